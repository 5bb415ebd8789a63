// gl_common.cuh -- device-side definitions shared by the kernels of the map
// optimiser (arXiv 2404.06926, Sec. III-A/III-C).  Nothing here is shared with
// the CPU oracle: constants and arithmetic are written out for the GPU alone.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gl {

// ---------------------------------------------------------------------------
// Constants.  The paper defers all rasteriser constants to 3DGS and prints
// none; these are the readings used throughout.
// ---------------------------------------------------------------------------
constexpr float kZNear = 0.2f;          // cull depth (m)
constexpr float kDilation = 0.3f;       // low-pass dilation added to Sigma' (px^2)
constexpr float kJacClamp = 1.3f;       // |x/z| <= 1.3 * tan(half FoV) in the EWA Jacobian
constexpr float kEigFloor = 0.1f;       // floor under the eigenvalue discriminant
constexpr float kRadiusSigmas = 3.0f;   // screen radius = ceil(3 sqrt(lambda_max))
constexpr float kAlphaMax = 0.99f;      // alpha cap
constexpr float kAlphaMin = 1.0f / 255.0f;  // alpha skip threshold
constexpr float kTransMin = 1e-4f;      // transmittance stop threshold

// Real SH normalisation factors (Condon-Shortley phase), degree <= 3.
constexpr float kSH0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kSH1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float kSH2a = 1.0925484305920792f;   // sqrt(15/pi)/2      xy, yz, xz
constexpr float kSH2b = 0.31539156525252005f;  // sqrt(5/pi)/4       2z^2-x^2-y^2
constexpr float kSH2c = 0.5462742152960396f;   // sqrt(15/pi)/4      x^2-y^2
constexpr float kSH3a = 0.5900435899266435f;   // sqrt(35/(2pi))/4   y(3x^2-y^2), x(x^2-3y^2)
constexpr float kSH3b = 2.890611442640554f;    // sqrt(105/pi)/2     xyz
constexpr float kSH3c = 0.4570457994644658f;   // sqrt(21/(2pi))/4   y(4z^2-x^2-y^2), x(..)
constexpr float kSH3d = 0.3731763325901154f;   // sqrt(7/pi)/4       z(2z^2-3x^2-3y^2)
constexpr float kSH3e = 1.445305721320277f;    // sqrt(105/pi)/4     z(x^2-y^2)

constexpr unsigned kFull = 0xffffffffu;

// Camera passed by value to kernels: world->camera x_c = R x_w + t, pinhole.
struct Cam {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int W, H;
};

// One view of a (possibly multi-view) step, read by the kernels from device
// memory.  Views are concatenated: raster tiles, 32x32 loss tiles and pixels
// of view v start at tile_base, ltile_base and pix_base.
struct ViewDesc {
    Cam cam;
    int TX, TY;              // raster tiles of the view
    int tile_base;           // global index of the view's first raster tile
    int ltile_base;          // global index of the view's first 32x32 loss tile
    long long pix_base;      // first pixel of the view in the concatenated images
    const float* target;     // loss target (H*W*3 RGB) or null
    float* E;                // exposure [A | b] (12) read by the loss; null = identity
    float* Em;               // Adam moments of E: m (12) then v (12); null = E not updated
    float e_bc1, e_bc2;      // exposure Adam bias corrections 1 - beta^t for this step
    float weight;            // weight of the view's loss in the step (1 / views)
    int pad;
};

// View of a global raster tile (views are few; linear search over the table).
__device__ __forceinline__ int view_of_tile(const ViewDesc* __restrict__ views, int V, int tile)
{
    int v = 0;
    while (v + 1 < V && views[v + 1].tile_base <= tile) v++;
    return v;
}

__device__ __forceinline__ int view_of_ltile(const ViewDesc* __restrict__ views, int V, int lt)
{
    int v = 0;
    while (v + 1 < V && views[v + 1].ltile_base <= lt) v++;
    return v;
}

// Read-only view of Gaussian parameters (device, one row-major array each).
struct GParams {
    const float* means;       // n*3
    const float* log_scales;  // n*3
    const float* quats;       // n*4 (w,x,y,z)
    const float* logits;      // n
    const float* sh;          // n*K*3
    int64_t n;
    int deg;
    int K;                    // (deg+1)^2
};

// Writable view (gradients, Adam moments, parameters updated in place).
struct GMut {
    float* means;
    float* log_scales;
    float* quats;
    float* logits;
    float* sh;
};

// ---------------------------------------------------------------------------
// Integer-deciding projection (Eq. 2-3): cull, radius, tile rectangle and
// depth key.  Every operation is an explicitly rounded float32 operation in
// a fixed order (no contraction), so the decision is reproducible.
// ---------------------------------------------------------------------------
struct Decision {
    float u, v, z;           // mu' and depth
    float a, b, c, det;      // Sigma' (dilated) and its determinant
    int r;                   // screen radius (px)
    int x0, y0, x1, y1;      // tile rectangle, half open
    float cA, cB, cC, ks;    // conic and the exact tile culling threshold (see tile_keep)
    float bc, ba;            // edge minimiser slopes -B/C, -B/A
};

__device__ __forceinline__ float fmr(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float far_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsr(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdr(float a, float b) { return __fdiv_rn(a, b); }

// exp of the decision path: x = k ln2 + r (ln2 as a 16-bit head plus tail),
// Taylor polynomial of exp(r) to degree 8 by Horner's rule, times 2^k -- a
// fixed sequence of correctly rounded float32 operations (no FP64, no
// contraction), accurate to a couple of ulp for |r| <= ln2/2.
__device__ __forceinline__ float expf_decision(float x)
{
    const float ln2_hi = 0.693145751953125f;
    const float ln2_lo = 1.42860682030941723212e-6f;
    const float k = rintf(__fmul_rn(x, 1.44269504088896340736f));
    const float r = __fsub_rn(__fsub_rn(x, __fmul_rn(k, ln2_hi)), __fmul_rn(k, ln2_lo));
    float p = 1.0f / 40320.0f;
    p = __fadd_rn(__fmul_rn(p, r), 1.0f / 5040.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f / 720.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f / 120.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f / 24.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f / 6.0f);
    p = __fadd_rn(__fmul_rn(p, r), 0.5f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    if (!(k >= -300.0f && k <= 300.0f)) return k > 0.0f ? __int_as_float(0x7f800000) : 0.0f;
    return ldexpf(p, (int)k);
}

// log of the decision path: x = m 2^e with m in [sqrt(1/2), sqrt(2)) from
// the bits, ln m = 2 atanh(s), s = (m - 1)/(m + 1), by its odd series to s^11
// (|s| <= 0.1716), then e ln2 with ln2 split as in expf_decision.
__device__ __forceinline__ float logf_decision(float x)
{
    if (!(x > 0.0f)) return __int_as_float(0xff800000);
    if (x == __int_as_float(0x7f800000)) return x;
    int e0 = 0;
    if (x < 1.17549435e-38f) { x = __fmul_rn(x, 16777216.0f); e0 = -24; }   // subnormal: scale by 2^24
    const unsigned bits = __float_as_uint(x);
    int e = (int)((bits >> 23) & 0xffu) - 126 + e0;
    float m = __uint_as_float((bits & 0x7fffffu) | 0x3f000000u);   // [0.5, 1)
    if (m < 0.70710678118654752f) { m = __fmul_rn(m, 2.0f); e -= 1; }
    const float ln2_hi = 0.693145751953125f;
    const float ln2_lo = 1.42860682030941723212e-6f;
    const float sv = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s2 = __fmul_rn(sv, sv);
    float p = (float)(2.0 / 11.0);
    p = __fadd_rn(__fmul_rn(p, s2), (float)(2.0 / 9.0));
    p = __fadd_rn(__fmul_rn(p, s2), (float)(2.0 / 7.0));
    p = __fadd_rn(__fmul_rn(p, s2), (float)(2.0 / 5.0));
    p = __fadd_rn(__fmul_rn(p, s2), (float)(2.0 / 3.0));
    p = __fadd_rn(__fmul_rn(p, s2), 2.0f);
    const float lm = __fmul_rn(p, sv);
    const float fe = (float)e;
    return __fadd_rn(__fmul_rn(fe, ln2_hi), __fadd_rn(__fmul_rn(fe, ln2_lo), lm));
}

// Exact tile culling (decision path): can the Gaussian reach alpha >= 1/255
// at a pixel centre of the tile whose centres span [X0, X0 + T1] x [Y0, Y0 +
// T1]?  q(d) = A dx^2 + 2 B dx dy + C dy^2 is convex, so off the rectangle
// its minimum lies on an edge, where the 1-D minimiser (dy = (-B/C) dx on
// x = const, dx = (-B/A) dy on y = const) is clamped to the edge; kept iff
// the minimum is <= ks = 2 ln(255 o) plus a slack of 2^-7
// (relative and absolute), so every dropped tile stays below the alpha
// threshold by far more than the per-pixel alpha's rounding.
__device__ __forceinline__ bool tile_keep(const Decision& D, float X0, float Y0, float T1)
{
    const float u = D.u, v = D.v, A = D.cA, B = D.cB, C = D.cC;
    const float dx0 = fsr(X0, u), dx1 = fsr(far_(X0, T1), u), dy0 = fsr(Y0, v), dy1 = fsr(far_(Y0, T1), v);
    if (dx0 <= 0.0f && dx1 >= 0.0f && dy0 <= 0.0f && dy1 >= 0.0f) return true;
    const float B2 = fmr(2.0f, B);
    float qmin = __int_as_float(0x7f800000);
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float dx = i ? dx1 : dx0;
        const float t = fminf(fmaxf(fmr(D.bc, dx), dy0), dy1);
        const float q = far_(far_(fmr(fmr(A, dx), dx), fmr(fmr(B2, dx), t)), fmr(fmr(C, t), t));
        qmin = fminf(qmin, q);
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float dy = i ? dy1 : dy0;
        const float t = fminf(fmaxf(fmr(D.ba, dy), dx0), dx1);
        const float q = far_(far_(fmr(fmr(A, t), t), fmr(fmr(B2, t), dy)), fmr(fmr(C, dy), dy));
        qmin = fminf(qmin, q);
    }
    return qmin <= D.ks;
}

__device__ __forceinline__ bool decide(const float mu[3], const float ls[3], const float q[4], float logit,
                                       const Cam& cam, int Ts, int TX, int TY, Decision& D)
{
    const float* R = cam.R;
    float x = far_(far_(far_(fmr(R[0], mu[0]), fmr(R[1], mu[1])), fmr(R[2], mu[2])), cam.t[0]);
    float y = far_(far_(far_(fmr(R[3], mu[0]), fmr(R[4], mu[1])), fmr(R[5], mu[2])), cam.t[1]);
    float z = far_(far_(far_(fmr(R[6], mu[0]), fmr(R[7], mu[1])), fmr(R[8], mu[2])), cam.t[2]);
    if (!(z > kZNear)) return false;
    float iz = fdr(1.0f, z);
    float xz = fmr(x, iz), yz = fmr(y, iz);
    float u = far_(fmr(cam.fx, xz), cam.cx);
    float v = far_(fmr(cam.fy, yz), cam.cy);
    if (!(fabsf(u) <= 3.0e38f) || !(fabsf(v) <= 3.0e38f)) return false;

    float s0 = expf_decision(ls[0]);
    float s1 = expf_decision(ls[1]);
    float s2 = expf_decision(ls[2]);
    float qq = far_(far_(far_(fmr(q[0], q[0]), fmr(q[1], q[1])), fmr(q[2], q[2])), fmr(q[3], q[3]));
    if (!(qq > 0.0f) || !(qq <= 3.0e38f)) return false;
    float inv = fdr(1.0f, __fsqrt_rn(qq));
    float w = fmr(q[0], inv), qx = fmr(q[1], inv), qy = fmr(q[2], inv), qz = fmr(q[3], inv);
    float r00 = fsr(1.0f, fmr(2.0f, far_(fmr(qy, qy), fmr(qz, qz))));
    float r01 = fmr(2.0f, fsr(fmr(qx, qy), fmr(w, qz)));
    float r02 = fmr(2.0f, far_(fmr(qx, qz), fmr(w, qy)));
    float r10 = fmr(2.0f, far_(fmr(qx, qy), fmr(w, qz)));
    float r11 = fsr(1.0f, fmr(2.0f, far_(fmr(qx, qx), fmr(qz, qz))));
    float r12 = fmr(2.0f, fsr(fmr(qy, qz), fmr(w, qx)));
    float r20 = fmr(2.0f, fsr(fmr(qx, qz), fmr(w, qy)));
    float r21 = fmr(2.0f, far_(fmr(qy, qz), fmr(w, qx)));
    float r22 = fsr(1.0f, fmr(2.0f, far_(fmr(qx, qx), fmr(qy, qy))));
    float M[9] = {fmr(r00, s0), fmr(r01, s1), fmr(r02, s2),
                  fmr(r10, s0), fmr(r11, s1), fmr(r12, s2),
                  fmr(r20, s0), fmr(r21, s1), fmr(r22, s2)};
    float S[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            S[i * 3 + j] = far_(far_(fmr(M[i * 3 + 0], M[j * 3 + 0]), fmr(M[i * 3 + 1], M[j * 3 + 1])),
                                fmr(M[i * 3 + 2], M[j * 3 + 2]));

    float limx = fmr(kJacClamp, fdr(fmr(0.5f, (float)cam.W), cam.fx));
    float limy = fmr(kJacClamp, fdr(fmr(0.5f, (float)cam.H), cam.fy));
    float cxz = fminf(fmaxf(xz, -limx), limx);
    float cyz = fminf(fmaxf(yz, -limy), limy);
    float j00 = fmr(cam.fx, iz);
    float j02 = fmr(-fmr(cam.fx, cxz), iz);
    float j11 = fmr(cam.fy, iz);
    float j12 = fmr(-fmr(cam.fy, cyz), iz);
    float T[6];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        T[k] = far_(fmr(j00, R[k]), fmr(j02, R[6 + k]));
        T[3 + k] = far_(fmr(j11, R[3 + k]), fmr(j12, R[6 + k]));
    }
    float U[6];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int k = 0; k < 3; k++)
            U[i * 3 + k] = far_(far_(fmr(T[i * 3 + 0], S[0 * 3 + k]), fmr(T[i * 3 + 1], S[1 * 3 + k])),
                                fmr(T[i * 3 + 2], S[2 * 3 + k]));
    float a = far_(far_(far_(fmr(U[0], T[0]), fmr(U[1], T[1])), fmr(U[2], T[2])), kDilation);
    float b = far_(far_(fmr(U[0], T[3]), fmr(U[1], T[4])), fmr(U[2], T[5]));
    float c = far_(far_(far_(fmr(U[3], T[3]), fmr(U[4], T[4])), fmr(U[5], T[5])), kDilation);
    float det = fsr(fmr(a, c), fmr(b, b));
    if (!(det > 0.0f)) return false;
    float mid = fmr(0.5f, far_(a, c));
    float lam = far_(mid, __fsqrt_rn(fmaxf(kEigFloor, fsr(fmr(mid, mid), det))));
    float r = ceilf(fmr(kRadiusSigmas, __fsqrt_rn(lam)));
    if (!(r >= 1.0f) || !(r <= 3.0e38f)) return false;

    float tsf = (float)Ts;
    float x0 = fminf(fmaxf(floorf(fdr(fsr(u, r), tsf)), 0.0f), (float)TX);
    float x1 = fminf(fmaxf(floorf(fdr(far_(far_(u, r), tsf - 1.0f), tsf)), 0.0f), (float)TX);
    float y0 = fminf(fmaxf(floorf(fdr(fsr(v, r), tsf)), 0.0f), (float)TY);
    float y1 = fminf(fmaxf(floorf(fdr(far_(far_(v, r), tsf - 1.0f), tsf)), 0.0f), (float)TY);
    D.x0 = (int)x0; D.y0 = (int)y0; D.x1 = (int)x1; D.y1 = (int)y1;
    if ((D.x1 - D.x0) * (D.y1 - D.y0) == 0) return false;
    D.r = (r > 2.0e9f) ? 2000000000 : (int)r;
    D.u = u; D.v = v; D.z = z;
    D.a = a; D.b = b; D.c = c; D.det = det;
    // exact tile culling inputs: conic and 2 ln(255 o) with slack
    const float og = fdr(1.0f, far_(1.0f, expf_decision(-logit)));
    const float kap = fmr(2.0f, logf_decision(fmr(255.0f, og)));
    D.cA = fdr(c, det);
    D.cB = fdr(-b, det);
    D.cC = fdr(a, det);
    D.ks = far_(kap, far_(fmr(kap, 0.0078125f), 0.0078125f));
    D.bc = fdr(-D.cB, D.cC);
    D.ba = fdr(-D.cB, D.cA);
    return true;
}

// The exact culling applies to rectangles of at most 64 tiles (a larger one
// keeps all its tiles, which is always allowed: it only costs instances).
constexpr int kCullMaxTiles = 64;

// Tiles of the rectangle the exact culling keeps; *mask gets them (bit i =
// the i-th tile in row-major order; all ones when nothing is culled).
__device__ __forceinline__ uint32_t kept_tiles(const Decision& D, int Ts, bool cull, unsigned long long* mask)
{
    const int area = (D.x1 - D.x0) * (D.y1 - D.y0);
    *mask = ~0ull;
    if (!cull || area > kCullMaxTiles) return (uint32_t)area;
    unsigned long long m = 0;
    const float T1 = (float)(Ts - 1);
    int i = 0;
    for (int ty = D.y0; ty < D.y1; ty++)
        for (int tx = D.x0; tx < D.x1; tx++, i++)
            if (tile_keep(D, (float)(tx * Ts), (float)(ty * Ts), T1)) m |= 1ull << i;
    *mask = m;
    return (uint32_t)__popcll(m);
}

// ---------------------------------------------------------------------------
// Real SH basis (degree <= 3) at a unit direction; optional gradient.
// ---------------------------------------------------------------------------
template <int DEG>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float Y[16])
{
    Y[0] = kSH0;
    if (DEG >= 1) { Y[1] = -kSH1 * y; Y[2] = kSH1 * z; Y[3] = -kSH1 * x; }
    if (DEG >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kSH2a * x * y;
        Y[5] = -kSH2a * y * z;
        Y[6] = kSH2b * (2.0f * zz - xx - yy);
        Y[7] = -kSH2a * x * z;
        Y[8] = kSH2c * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -kSH3a * y * (3.0f * xx - yy);
            Y[10] = kSH3b * x * y * z;
            Y[11] = -kSH3c * y * (4.0f * zz - xx - yy);
            Y[12] = kSH3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
            Y[13] = -kSH3c * x * (4.0f * zz - xx - yy);
            Y[14] = kSH3e * z * (xx - yy);
            Y[15] = -kSH3a * x * (xx - 3.0f * yy);
        }
    }
}

// g += sum_k c_k grad Y_k(x, y, z) with c_k = sum_c sh[3k + c] w[c] (dir treated
// as unconstrained); the basis gradient is never materialised.
template <int DEG>
__device__ __forceinline__ void sh_grad_acc(float x, float y, float z, const float* __restrict__ sh,
                                            const float w[3], float g[3])
{
#define GL_CF(k) (sh[3 * (k)] * w[0] + sh[3 * (k) + 1] * w[1] + sh[3 * (k) + 2] * w[2])
    if (DEG >= 1) {
        g[1] -= kSH1 * GL_CF(1);
        g[2] += kSH1 * GL_CF(2);
        g[0] -= kSH1 * GL_CF(3);
    }
    if (DEG >= 2) {
        float c = GL_CF(4);
        g[0] += c * kSH2a * y; g[1] += c * kSH2a * x;
        c = GL_CF(5);
        g[1] -= c * kSH2a * z; g[2] -= c * kSH2a * y;
        c = GL_CF(6);
        g[0] -= c * 2.0f * kSH2b * x; g[1] -= c * 2.0f * kSH2b * y; g[2] += c * 4.0f * kSH2b * z;
        c = GL_CF(7);
        g[0] -= c * kSH2a * z; g[2] -= c * kSH2a * x;
        c = GL_CF(8);
        g[0] += c * 2.0f * kSH2c * x; g[1] -= c * 2.0f * kSH2c * y;
    }
    if (DEG >= 3) {
        const float xx = x * x, yy = y * y, zz = z * z;
        float c = GL_CF(9);
        g[0] -= c * kSH3a * 6.0f * x * y; g[1] -= c * kSH3a * (3.0f * xx - 3.0f * yy);
        c = GL_CF(10);
        g[0] += c * kSH3b * y * z; g[1] += c * kSH3b * x * z; g[2] += c * kSH3b * x * y;
        c = GL_CF(11);
        g[0] += c * kSH3c * 2.0f * x * y; g[1] -= c * kSH3c * (4.0f * zz - xx - 3.0f * yy);
        g[2] -= c * kSH3c * 8.0f * y * z;
        c = GL_CF(12);
        g[0] -= c * kSH3d * 6.0f * x * z; g[1] -= c * kSH3d * 6.0f * y * z;
        g[2] += c * kSH3d * (6.0f * zz - 3.0f * xx - 3.0f * yy);
        c = GL_CF(13);
        g[0] -= c * kSH3c * (4.0f * zz - 3.0f * xx - yy); g[1] += c * kSH3c * 2.0f * x * y;
        g[2] -= c * kSH3c * 8.0f * x * z;
        c = GL_CF(14);
        g[0] += c * kSH3e * 2.0f * x * z; g[1] -= c * kSH3e * 2.0f * y * z; g[2] += c * kSH3e * (xx - yy);
        c = GL_CF(15);
        g[0] -= c * kSH3a * (3.0f * xx - 3.0f * yy); g[1] += c * kSH3a * 6.0f * x * y;
    }
#undef GL_CF
}

// ---------------------------------------------------------------------------
// The screen-space mean mu' = pi(R mu + t) (Eq. 2) for rendering, in
// double-float arithmetic: a value is an unevaluated sum hi + lo of two
// floats, built from the error-free transformations TwoSum (Knuth) and
// TwoProd by fused multiply-add (the method of Dekker, 1971).  World
// coordinates of tens to hundreds of metres cancel in R mu + t, and a float
// product loses up to ~1e-4 px of the mean at 1280 px; the double-float
// result is exact to ~1e-12 px, so a pixel's offset from the mean can be
// formed to float precision relative to its tile (see the record permute).
// The decision path (decide) keeps its own rounded float mean.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// (ah + al) + (bh + bl)
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& sh, float& sl)
{
    float s, e;
    two_sum(ah, bh, s, e);
    two_sum(s, __fadd_rn(e, __fadd_rn(al, bl)), sh, sl);
}

// (ah + al) * b
__device__ __forceinline__ void df_mul_f(float ah, float al, float b, float& ph, float& pl)
{
    float p, e;
    two_prod(ah, b, p, e);
    two_sum(p, __fmaf_rn(al, b, e), ph, pl);
}

// (ah + al) / (bh + bl): the float quotient plus one correction from the
// remainder a - q b, formed with TwoProd
__device__ __forceinline__ void df_div(float ah, float al, float bh, float bl, float& qh, float& ql)
{
    const float q1 = __fdiv_rn(ah, bh);
    float p, e;
    two_prod(q1, bh, p, e);
    float rh, re;
    two_sum(ah, -p, rh, re);
    const float r = __fadd_rn(__fsub_rn(__fadd_rn(rh, __fadd_rn(re, al)), e), -__fmul_rn(q1, bl));
    two_sum(q1, __fdiv_rn(r, bh), qh, ql);
}

// mu' as (u_hi + u_lo, v_hi + v_lo); z > 0 is known (the decision passed)
__device__ __forceinline__ void mean2d_df(const float mu[3], const Cam& cam, float& uh, float& ul, float& vh,
                                          float& vl)
{
    float c[3][2];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        float h, l, ph, pl;
        two_prod(cam.R[3 * i], mu[0], h, l);
        two_prod(cam.R[3 * i + 1], mu[1], ph, pl);
        df_add(h, l, ph, pl, h, l);
        two_prod(cam.R[3 * i + 2], mu[2], ph, pl);
        df_add(h, l, ph, pl, h, l);
        df_add(h, l, cam.t[i], 0.0f, c[i][0], c[i][1]);
    }
    float qh, ql;
    df_div(c[0][0], c[0][1], c[2][0], c[2][1], qh, ql);
    df_mul_f(qh, ql, cam.fx, qh, ql);
    df_add(qh, ql, cam.cx, 0.0f, uh, ul);
    df_div(c[1][0], c[1][1], c[2][0], c[2][1], qh, ql);
    df_mul_f(qh, ql, cam.fy, qh, ql);
    df_add(qh, ql, cam.cy, 0.0f, vh, vl);
}

// ---------------------------------------------------------------------------
// Per-pair blending weight (Eq. 4) shared by the forward and the backward
// raster kernels, evaluated in the log2 domain:
//   e = log2(o exp(power)) = A' dx^2 + C' dy^2 + B' dx dy + log2(o),
// with A' = -A log2(e)/2, C' = -C log2(e)/2, B' = -B log2(e) precomputed per
// Gaussian.  The pair is skipped when e < log2(1/255) (alpha below 1/255) or
// when e > log2(o) (power > 0, possible only through rounding).  Explicitly
// rounded operations keep the decisions of the two kernels identical.
// Records as the raster kernels read them (sorted-instance order): r0 =
// (u, v, A', C') with (u, v) relative to the origin of the instance's tile,
// r1 = (B', log2 o, depth, -); (px, py) are tile-relative pixel coordinates.
// ---------------------------------------------------------------------------
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLog2AlphaMin = -7.994353436858858f;   // log2(1/255)

__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ bool pair_eval(const float4 r0, const float4 r1, float px, float py,
                                          float& dx, float& dy, float& alpha, bool& capped)
{
    dx = __fsub_rn(r0.x, px);
    dy = __fsub_rn(r0.y, py);
    const float e = __fmaf_rn(__fmul_rn(r0.z, dx), dx,
                              __fmaf_rn(__fmul_rn(r0.w, dy), dy, __fmaf_rn(__fmul_rn(r1.x, dx), dy, r1.y)));
    if (!(e >= kLog2AlphaMin) || e > r1.y) return false;
    const float araw = ex2_approx(e);
    capped = araw >= kAlphaMax;
    alpha = fminf(kAlphaMax, araw);
    return true;
}

// pair_eval without the early exit: alpha and capped are computed whatever
// the outcome (meaningful only when it returns true).
__device__ __forceinline__ bool pair_eval_nb(const float4 r0, const float4 r1, float px, float py, float& dx,
                                             float& dy, float& alpha, bool& capped)
{
    dx = __fsub_rn(r0.x, px);
    dy = __fsub_rn(r0.y, py);
    const float e = __fmaf_rn(__fmul_rn(r0.z, dx), dx,
                              __fmaf_rn(__fmul_rn(r0.w, dy), dy, __fmaf_rn(__fmul_rn(r1.x, dx), dy, r1.y)));
    const float araw = ex2_approx(e);
    capped = araw >= kAlphaMax;
    alpha = fminf(kAlphaMax, araw);
    return e >= kLog2AlphaMin && !(e > r1.y);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

}  // namespace gl
