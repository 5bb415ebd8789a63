// gl_params.cu -- backward of the projection and colour (Eq. 1-3, SH) from the
// per-instance screen-space gradients to every Gaussian attribute and to the
// camera pose, and the fused (sparse) Adam update (Sec. III-D 2).
//
// One thread per Gaussian.  It sums the gradients of its (Gaussian, tile)
// instances -- contiguous, because instances are emitted per Gaussian --
// recomputes the forward geometry in registers, applies the chain rule and
// either writes the gradients (differentiable API) or updates the parameters
// and both Adam moments in place, so the 59-float gradient never reaches
// memory on the optimisation path.
#include "gl_internal.h"

#include <algorithm>

namespace gl {

namespace {

constexpr int kThreads = 128;
constexpr int kUnroll = 4;   // float4 loads per thread in flight in the Adam pass
constexpr int kNG = 10;

struct Geo {
    float x, y, z, iz;
    float s[3], qn[4], qnorm, Rq[9], M[9], Sig[9];
    float J00, J02, J11, J12;
    bool clx, cly;
    float T[6], a, b, c, A, B, C;
    float o;
    float dir[3], dnorm;
};

__device__ __forceinline__ void geometry(const float mu[3], const float ls[3], const float q[4],
                                         float logit, const Cam& cam, Geo& G)
{
    const float* R = cam.R;
    G.x = R[0] * mu[0] + R[1] * mu[1] + R[2] * mu[2] + cam.t[0];
    G.y = R[3] * mu[0] + R[4] * mu[1] + R[5] * mu[2] + cam.t[1];
    G.z = R[6] * mu[0] + R[7] * mu[1] + R[8] * mu[2] + cam.t[2];
    G.iz = 1.0f / G.z;
    for (int i = 0; i < 3; i++) G.s[i] = expf(ls[i]);
    float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    G.qnorm = sqrtf(qq);
    float inv = 1.0f / G.qnorm;
    for (int i = 0; i < 4; i++) G.qn[i] = q[i] * inv;
    const float w = G.qn[0], x = G.qn[1], y = G.qn[2], z = G.qn[3];
    G.Rq[0] = 1.f - 2.f * (y * y + z * z); G.Rq[1] = 2.f * (x * y - w * z); G.Rq[2] = 2.f * (x * z + w * y);
    G.Rq[3] = 2.f * (x * y + w * z); G.Rq[4] = 1.f - 2.f * (x * x + z * z); G.Rq[5] = 2.f * (y * z - w * x);
    G.Rq[6] = 2.f * (x * z - w * y); G.Rq[7] = 2.f * (y * z + w * x); G.Rq[8] = 1.f - 2.f * (x * x + y * y);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) G.M[i * 3 + j] = G.Rq[i * 3 + j] * G.s[j];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            G.Sig[i * 3 + j] = G.M[i * 3] * G.M[j * 3] + G.M[i * 3 + 1] * G.M[j * 3 + 1] + G.M[i * 3 + 2] * G.M[j * 3 + 2];
    const float limx = kJacClamp * (0.5f * (float)cam.W / cam.fx);
    const float limy = kJacClamp * (0.5f * (float)cam.H / cam.fy);
    const float xz = G.x * G.iz, yz = G.y * G.iz;
    G.clx = xz < -limx || xz > limx;
    G.cly = yz < -limy || yz > limy;
    const float cxz = fminf(fmaxf(xz, -limx), limx), cyz = fminf(fmaxf(yz, -limy), limy);
    G.J00 = cam.fx * G.iz;
    G.J02 = -cam.fx * cxz * G.iz;
    G.J11 = cam.fy * G.iz;
    G.J12 = -cam.fy * cyz * G.iz;
    for (int k = 0; k < 3; k++) {
        G.T[k] = G.J00 * R[k] + G.J02 * R[6 + k];
        G.T[3 + k] = G.J11 * R[3 + k] + G.J12 * R[6 + k];
    }
    float U[6];
    for (int i = 0; i < 2; i++)
        for (int k = 0; k < 3; k++)
            U[i * 3 + k] = G.T[i * 3] * G.Sig[k] + G.T[i * 3 + 1] * G.Sig[3 + k] + G.T[i * 3 + 2] * G.Sig[6 + k];
    G.a = U[0] * G.T[0] + U[1] * G.T[1] + U[2] * G.T[2] + kDilation;
    G.b = U[0] * G.T[3] + U[1] * G.T[4] + U[2] * G.T[5];
    G.c = U[3] * G.T[3] + U[4] * G.T[4] + U[5] * G.T[5] + kDilation;
    const float idet = 1.0f / (G.a * G.c - G.b * G.b);
    G.A = G.c * idet;
    G.B = -G.b * idet;
    G.C = G.a * idet;
    G.o = 1.0f / (1.0f + expf(-logit));
    const float cw0 = -(R[0] * cam.t[0] + R[3] * cam.t[1] + R[6] * cam.t[2]);
    const float cw1 = -(R[1] * cam.t[0] + R[4] * cam.t[1] + R[7] * cam.t[2]);
    const float cw2 = -(R[2] * cam.t[0] + R[5] * cam.t[1] + R[8] * cam.t[2]);
    const float d0 = mu[0] - cw0, d1 = mu[1] - cw1, d2 = mu[2] - cw2;
    G.dnorm = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    const float idn = 1.0f / G.dnorm;
    G.dir[0] = d0 * idn; G.dir[1] = d1 * idn; G.dir[2] = d2 * idn;
}

// Hint the L2 to fetch [p, p + bytes) (the 16-byte aligned part of it) with
// one bulk prefetch; nothing waits for it.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes)
{
    const uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
    const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
    if (e > a) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(e - a)) : "memory");
}

// Shared-memory row stride of an array of WIDTH floats per Gaussian: rows of
// an even number of float4 get one float4 of padding, so that the float4
// reads of a quarter warp (8 rows) fall in distinct banks.
template <int WIDTH>
constexpr int staged_stride() { return (WIDTH % 4 == 0 && (WIDTH / 4) % 2 == 0) ? WIDTH + 4 : WIDTH; }

// Copy the block's rows [g0, g0 + cnt) of one parameter array into shared
// memory at the staged stride; float4 loads where rows allow them.
template <int WIDTH>
__device__ __forceinline__ void stage_rows(const float* __restrict__ P, int64_t g0, int cnt, float* __restrict__ dst)
{
    constexpr int S = staged_stride<WIDTH>();
    const float* src = P + (size_t)g0 * WIDTH;
    const int ne = cnt * WIDTH;
    if constexpr (WIDTH % 4 == 0) {
        constexpr int R4 = WIDTH / 4;
        const float4* s4 = reinterpret_cast<const float4*>(src);
        float4* d4 = reinterpret_cast<float4*>(dst);
        for (int f = threadIdx.x; f < ne / 4; f += kThreads) d4[(f / R4) * (S / 4) + f % R4] = s4[f];
    } else {
        // S == WIDTH: the span is copied as is
        const int nv = ne / 4;
        const float4* s4 = reinterpret_cast<const float4*>(src);
        float4* d4 = reinterpret_cast<float4*>(dst);
        for (int f = threadIdx.x; f < nv; f += kThreads) d4[f] = s4[f];
        for (int e = 4 * nv + threadIdx.x; e < ne; e += kThreads) dst[e] = src[e];
    }
}

// p -= lr (m / bc1) / (sqrt(v / bc2) + eps), with 1/bc1 and 1/sqrt(bc2)
// precomputed for the step: the same update with one square root and one
// fast division per element.
__device__ __forceinline__ void adam1(float& p, float& m, float& v, float g, float lr, const AdamArgs& a)
{
    m = a.b1 * m + (1.0f - a.b1) * g;
    v = a.b2 * v + (1.0f - a.b2) * g * g;
    // sqrt(v) as v * rsqrt(v) (the hardware reciprocal square root, a few
    // ulp), 0 at v = 0
    const float sv = v > 0.0f ? v * rsqrtf(v) : 0.0f;
    p -= __fdividef(lr * a.ibc1 * m, sv * a.isbc2 + a.eps);
}

// Block-cooperative pass over one parameter array of the block's Gaussians
// (a contiguous span of cnt * WIDTH floats, 16-byte aligned because blocks
// start at multiples of 128 Gaussians): MODE 0 writes the gradient rows
// (sR, stride NR, this array's columns from off), MODE 1 applies Adam to the
// parameters staged in shared memory (sP, rows at the staged stride) and
// writes them back with the moments (the first three floats of a row take
// lr0, the SH DC band; the rest lr).  Rows flagged off in upd are left
// untouched (MODE 1).  Rows of a multiple of 4 floats go by float4, a row
// quarter per thread; other widths element by element.  kUnroll accesses per
// thread are in flight.
template <int MODE, int WIDTH, int NR>
__device__ __forceinline__ void coop(float* __restrict__ P, float* __restrict__ Mm, float* __restrict__ Vv,
                                     int64_t g0, int cnt, const float* __restrict__ sR, int off,
                                     const float* __restrict__ sP, const uint8_t* __restrict__ upd, float lr,
                                     float lr0, const AdamArgs& ad)
{
    constexpr int S = staged_stride<WIDTH>();
    const size_t base = (size_t)g0 * WIDTH;
    if constexpr (WIDTH % 4 == 0) {
        constexpr int R4 = WIDTH / 4;
        const int nv = cnt * R4;
        float4* P4 = reinterpret_cast<float4*>(P + base);
        float4* M4 = reinterpret_cast<float4*>(Mm + base);
        float4* V4 = reinterpret_cast<float4*>(Vv + base);
        const float4* S4 = reinterpret_cast<const float4*>(sP);
        for (int f0 = threadIdx.x; f0 < nv; f0 += kUnroll * kThreads) {
            float4 pp[kUnroll], mm[kUnroll], vv[kUnroll];
            int row[kUnroll], c4[kUnroll];
            bool ok[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                const int f = f0 + u * kThreads;
                row[u] = f / R4;
                c4[u] = f - row[u] * R4;
                ok[u] = f < nv && (MODE == 0 || upd[row[u]]);
                if (ok[u] && MODE == 1) {
                    mm[u] = M4[f];
                    vv[u] = V4[f];
                    pp[u] = S4[row[u] * (S / 4) + c4[u]];
                }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                if (!ok[u]) continue;
                const int f = f0 + u * kThreads;
                const float* gr = sR + row[u] * NR + off + 4 * c4[u];
                if (MODE == 0) {
                    P4[f] = make_float4(gr[0], gr[1], gr[2], gr[3]);
                } else {
                    float* pa = &pp[u].x;
                    float* ma = &mm[u].x;
                    float* va = &vv[u].x;
#pragma unroll
                    for (int e = 0; e < 4; e++) adam1(pa[e], ma[e], va[e], gr[e], 4 * c4[u] + e < 3 ? lr0 : lr, ad);
                    P4[f] = pp[u];
                    M4[f] = mm[u];
                    V4[f] = vv[u];
                }
            }
        }
    } else {
        const int ne = cnt * WIDTH;
        for (int e0 = threadIdx.x; e0 < ne; e0 += kUnroll * kThreads) {
            float pv[kUnroll], mv[kUnroll], vv[kUnroll];
            int row[kUnroll], w[kUnroll];
            bool ok[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                const int e = e0 + u * kThreads;
                row[u] = e / WIDTH;
                w[u] = e - row[u] * WIDTH;
                ok[u] = e < ne && (MODE == 0 || upd[row[u]]);
                if (ok[u] && MODE == 1) {
                    mv[u] = Mm[base + e];
                    vv[u] = Vv[base + e];
                    pv[u] = sP[row[u] * S + w[u]];
                }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                if (!ok[u]) continue;
                const int e = e0 + u * kThreads;
                const float gr = sR[row[u] * NR + off + w[u]];
                if (MODE == 0) {
                    P[base + e] = gr;
                } else {
                    adam1(pv[u], mv[u], vv[u], gr, w[u] < 3 ? lr0 : lr, ad);
                    P[base + e] = pv[u];
                    Mm[base + e] = mv[u];
                    Vv[base + e] = vv[u];
                }
            }
        }
    }
}

// Shared memory of k_params_bwd (floats): the gradient rows (odd stride NR),
// then the block's staged parameter rows (means, log-scales, quaternions,
// logits, SH at their staged strides), each part 16-byte aligned.
template <int DEG>
struct ParamsSmem {
    static constexpr int KF = (DEG + 1) * (DEG + 1) * 3;   // SH floats per Gaussian
    static constexpr int NR = 11 + KF + ((11 + KF) % 2 == 0 ? 1 : 0);
    static constexpr int SHS = staged_stride<KF>();
    static constexpr int R = (kThreads * NR + 3) / 4 * 4;
    static constexpr int MU = R, LS = MU + kThreads * 3, Q = LS + kThreads * 3, LG = Q + kThreads * 4,
                         SH = LG + kThreads, END = SH + kThreads * SHS;
    static constexpr size_t bytes = sizeof(float) * (size_t)END;
};

template <int DEG, int MODE>
__global__ void __launch_bounds__(kThreads, 3)
k_params_bwd(GParams p, const ViewDesc* __restrict__ views, int V, const int* __restrict__ radius,
             const float* __restrict__ g2d, GMut out, AdamArgs ad, float* __restrict__ pose_part)
{
    using SM = ParamsSmem<DEG>;
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int KF = SM::KF;
    // one row of gradients per Gaussian of the block: means 3, log-scales 3,
    // quaternion 4, logit 1, SH KF (odd stride against bank conflicts); the
    // Adam update then streams every parameter array with coalesced accesses
    constexpr int NR = SM::NR;
    if (MODE == 1) {
        // a step whose binning overflowed its buffers updates nothing (it is re-run)
        if (ad.abort && ad.abort[1]) return;
        if (ad.bc) { ad.ibc1 = ad.bc[0]; ad.isbc2 = ad.bc[1]; }
    }
    extern __shared__ float4 smem4[];
    float* smf = reinterpret_cast<float*>(smem4);
    float* sR = smf;
    float* sMu = smf + SM::MU;
    float* sLs = smf + SM::LS;
    float* sQ = smf + SM::Q;
    float* sLg = smf + SM::LG;
    float* sSH = smf + SM::SH;
    __shared__ uint8_t sUpd[kThreads];
    const int64_t g0 = blockIdx.x * (int64_t)kThreads;
    const int64_t g = g0 + threadIdx.x;
    const int cnt = (int)min((int64_t)kThreads, p.n - g0);
    // the moments and screen-space gradients of the block head for the L2
    // while its parameters are staged and its geometry is recomputed
    if (threadIdx.x == 0) {
        if (MODE == 1) {
            const size_t c4 = sizeof(float) * (size_t)cnt;
            prefetch_l2(ad.m.means + 3 * g0, 3 * c4);
            prefetch_l2(ad.v.means + 3 * g0, 3 * c4);
            prefetch_l2(ad.m.log_scales + 3 * g0, 3 * c4);
            prefetch_l2(ad.v.log_scales + 3 * g0, 3 * c4);
            prefetch_l2(ad.m.quats + 4 * g0, 4 * c4);
            prefetch_l2(ad.v.quats + 4 * g0, 4 * c4);
            prefetch_l2(ad.m.logits + g0, c4);
            prefetch_l2(ad.v.logits + g0, c4);
            prefetch_l2(ad.m.sh + (size_t)KF * g0, KF * c4);
            prefetch_l2(ad.v.sh + (size_t)KF * g0, KF * c4);
        }
        for (int vw = 0; vw < V; vw++) {
            prefetch_l2(g2d + ((size_t)vw * p.n + g0) * kNG, sizeof(float) * kNG * (size_t)cnt);
            prefetch_l2(radius + (size_t)vw * p.n + g0, sizeof(int) * (size_t)cnt);
        }
    }
    stage_rows<3>(p.means, g0, cnt, sMu);
    stage_rows<3>(p.log_scales, g0, cnt, sLs);
    stage_rows<4>(p.quats, g0, cnt, sQ);
    stage_rows<1>(p.logits, g0, cnt, sLg);
    stage_rows<KF>(p.sh, g0, cnt, sSH);
    __syncthreads();
    float pose[6] = {0, 0, 0, 0, 0, 0};
    const bool valid = g < p.n;
    bool vis = false, first = true;

    float gm[3] = {0, 0, 0}, gl3[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, glg = 0.0f;
    float* dsh = sR + threadIdx.x * NR + 11;   // this Gaussian's SH gradient, summed over its views in place

    // every view the Gaussian is visible in contributes (window steps sum them)
    for (int vw = 0; vw < V && valid; vw++) {
    const int64_t tv = (int64_t)vw * p.n + g;
    if (radius[tv] <= 0) continue;
    vis = true;
    const Cam cam = views[vw].cam;
    float grgb[3] = {0, 0, 0};
    {
        float Y[16];
        const int r = threadIdx.x;
        float mu[3] = {sMu[3 * r], sMu[3 * r + 1], sMu[3 * r + 2]};
        float ls[3] = {sLs[3 * r], sLs[3 * r + 1], sLs[3 * r + 2]};
        const float4 q4 = reinterpret_cast<const float4*>(sQ)[r];
        float q[4] = {q4.x, q4.y, q4.z, q4.w};
        Geo G;
        geometry(mu, ls, q, sLg[r], cam, G);

        // screen-space gradients of this Gaussian, accumulated by the raster backward
        float s[kNG];
        for (int k = 0; k < kNG; k++) s[k] = g2d[(size_t)tv * kNG + k];
        const float du = -G.A * s[4] - G.B * s[5];
        const float dv = -G.C * s[5] - G.B * s[4];
        const float dA = -0.5f * s[6], dB = -s[7], dC = -0.5f * s[8];
        const float dop = s[3] / G.o;
        const float dz = s[9];

        // opacity
        glg += dop * G.o * (1.0f - G.o);

        // colour -> SH and view direction (clamped channels pass no gradient)
        sh_eval<DEG>(G.dir[0], G.dir[1], G.dir[2], Y);
        const float* sh = sSH + threadIdx.x * SM::SHS;
        float raw[3] = {0.5f, 0.5f, 0.5f};
        for (int k = 0; k < K; k++)
            for (int c = 0; c < 3; c++) raw[c] += Y[k] * sh[3 * k + c];
        for (int c = 0; c < 3; c++) grgb[c] = raw[c] < 0.0f ? 0.0f : s[c];
        // dL/dsh_k = Y_k dL/drgb (the first view writes the row)
#pragma unroll
        for (int k = 0; k < K; k++)
#pragma unroll
            for (int c = 0; c < 3; c++) dsh[3 * k + c] = (first ? 0.0f : dsh[3 * k + c]) + Y[k] * grgb[c];
        first = false;
        float gdir[3] = {0, 0, 0};
        if (DEG > 0) sh_grad_acc<DEG>(G.dir[0], G.dir[1], G.dir[2], sh, grgb, gdir);
        const float dd = G.dir[0] * gdir[0] + G.dir[1] * gdir[1] + G.dir[2] * gdir[2];
        float gdu[3];
        for (int j = 0; j < 3; j++) gdu[j] = (gdir[j] - G.dir[j] * dd) / G.dnorm;
        for (int j = 0; j < 3; j++) gm[j] += gdu[j];
        const float* R = cam.R;
        for (int i = 0; i < 3; i++) pose[i] += R[i * 3] * gdu[0] + R[i * 3 + 1] * gdu[1] + R[i * 3 + 2] * gdu[2];

        // conic -> Sigma' (a, b, c), written with the conic to avoid det^2
        const float A = G.A, B = G.B, C = G.C;
        const float ga = -A * A * dA - A * B * dB - B * B * dC;
        const float gb = -2.f * A * B * dA - (A * C + B * B) * dB - 2.f * B * C * dC;
        const float gc = -B * B * dA - B * C * dB - C * C * dC;
        const float Gm[4] = {ga, 0.5f * gb, 0.5f * gb, gc};
        // Sigma' = T Sigma T^T
        float gSig[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                const float t0i = G.T[i], t1i = G.T[3 + i], t0j = G.T[j], t1j = G.T[3 + j];
                gSig[i * 3 + j] = t0i * (Gm[0] * t0j + Gm[1] * t1j) + t1i * (Gm[2] * t0j + Gm[3] * t1j);
            }
        float TS[6];
        for (int r = 0; r < 2; r++)
            for (int j = 0; j < 3; j++)
                TS[r * 3 + j] = G.T[r * 3] * G.Sig[j] + G.T[r * 3 + 1] * G.Sig[3 + j] + G.T[r * 3 + 2] * G.Sig[6 + j];
        float gT[6];
        for (int r = 0; r < 2; r++)
            for (int j = 0; j < 3; j++)
                gT[r * 3 + j] = 2.f * (Gm[r * 2] * TS[j] + Gm[r * 2 + 1] * TS[3 + j]);
        // Sigma = M M^T, M = Rq diag(s)
        float gRq[9];
        for (int j = 0; j < 3; j++) {
            float acc = 0.0f;
            for (int i = 0; i < 3; i++) {
                const float gMij = 2.f * (gSig[i * 3] * G.M[j] + gSig[i * 3 + 1] * G.M[3 + j] + gSig[i * 3 + 2] * G.M[6 + j]);
                acc += gMij * G.Rq[i * 3 + j];
                gRq[i * 3 + j] = gMij * G.s[j];
            }
            gl3[j] += acc * G.s[j];
        }
        {
            const float w = G.qn[0], x = G.qn[1], y = G.qn[2], z = G.qn[3];
            float gn[4];
            gn[0] = 2.f * (-z * gRq[1] + y * gRq[2] + z * gRq[3] - x * gRq[5] - y * gRq[6] + x * gRq[7]);
            gn[1] = 2.f * (y * gRq[1] + z * gRq[2] + y * gRq[3] - 2.f * x * gRq[4] - w * gRq[5]
                           + z * gRq[6] + w * gRq[7] - 2.f * x * gRq[8]);
            gn[2] = 2.f * (-2.f * y * gRq[0] + x * gRq[1] + w * gRq[2] + x * gRq[3] + z * gRq[5]
                           - w * gRq[6] + z * gRq[7] - 2.f * y * gRq[8]);
            gn[3] = 2.f * (-2.f * z * gRq[0] - w * gRq[1] + x * gRq[2] + w * gRq[3] - 2.f * z * gRq[4]
                           + y * gRq[5] + x * gRq[6] + y * gRq[7]);
            const float qd = w * gn[0] + x * gn[1] + y * gn[2] + z * gn[3];
            for (int i = 0; i < 4; i++) gq[i] += (gn[i] - G.qn[i] * qd) / G.qnorm;
        }
        // T = J W
        float gJ00 = 0, gJ02 = 0, gJ11 = 0, gJ12 = 0;
        for (int k = 0; k < 3; k++) {
            gJ00 += gT[k] * R[k];
            gJ02 += gT[k] * R[6 + k];
            gJ11 += gT[3 + k] * R[3 + k];
            gJ12 += gT[3 + k] * R[6 + k];
        }
        // camera-space mean through mu', J and the depth output
        const float x = G.x, y = G.y, z = G.z, iz = G.iz, iz2 = iz * iz;
        float gmc[3];
        gmc[0] = du * cam.fx * iz;
        gmc[1] = dv * cam.fy * iz;
        gmc[2] = -(du * cam.fx * x + dv * cam.fy * y) * iz2 + dz;
        gmc[2] += -(gJ00 * cam.fx + gJ11 * cam.fy) * iz2;
        if (!G.clx) { gmc[0] += -gJ02 * cam.fx * iz2; gmc[2] += 2.f * gJ02 * cam.fx * x * iz2 * iz; }
        else { gmc[2] += -gJ02 * G.J02 * iz; }
        if (!G.cly) { gmc[1] += -gJ12 * cam.fy * iz2; gmc[2] += 2.f * gJ12 * cam.fy * y * iz2 * iz; }
        else { gmc[2] += -gJ12 * G.J12 * iz; }
        for (int j = 0; j < 3; j++) gm[j] += R[j] * gmc[0] + R[3 + j] * gmc[1] + R[6 + j] * gmc[2];
        pose[0] += gmc[0]; pose[1] += gmc[1]; pose[2] += gmc[2];
        pose[3] += y * gmc[2] - z * gmc[1];
        pose[4] += z * gmc[0] - x * gmc[2];
        pose[5] += x * gmc[1] - y * gmc[0];
        // dW = phi^ W: P = W gW^T with gW = J^T gT
        float gW[9];
        for (int k = 0; k < 3; k++) {
            gW[0 * 3 + k] = G.J00 * gT[k];
            gW[1 * 3 + k] = G.J11 * gT[3 + k];
            gW[2 * 3 + k] = G.J02 * gT[k] + G.J12 * gT[3 + k];
        }
        float P[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                P[i * 3 + j] = R[i * 3] * gW[j * 3] + R[i * 3 + 1] * gW[j * 3 + 1] + R[i * 3 + 2] * gW[j * 3 + 2];
        pose[3] += P[5] - P[7];
        pose[4] += P[6] - P[2];
        pose[5] += P[1] - P[3];
    }
    }
    if (!vis)
        for (int k = 0; k < KF; k++) dsh[k] = 0.0f;

    const bool upd = valid && (MODE == 0 || !ad.sparse || vis);
    sUpd[threadIdx.x] = upd ? 1 : 0;
    {
        float* row = sR + threadIdx.x * NR;
        row[0] = gm[0]; row[1] = gm[1]; row[2] = gm[2];
        row[3] = gl3[0]; row[4] = gl3[1]; row[5] = gl3[2];
        row[6] = gq[0]; row[7] = gq[1]; row[8] = gq[2]; row[9] = gq[3];
        row[10] = glg;
    }
    __syncthreads();
    if (cnt > 0) {
        coop<MODE, 3, NR>(out.means, ad.m.means, ad.v.means, g0, cnt, sR, 0, sMu, sUpd, ad.lr_pos, ad.lr_pos, ad);
        coop<MODE, 3, NR>(out.log_scales, ad.m.log_scales, ad.v.log_scales, g0, cnt, sR, 3, sLs, sUpd, ad.lr_scale,
                          ad.lr_scale, ad);
        coop<MODE, 4, NR>(out.quats, ad.m.quats, ad.v.quats, g0, cnt, sR, 6, sQ, sUpd, ad.lr_rot, ad.lr_rot, ad);
        coop<MODE, 1, NR>(out.logits, ad.m.logits, ad.v.logits, g0, cnt, sR, 10, sLg, sUpd, ad.lr_op, ad.lr_op,
                          ad);
        coop<MODE, KF, NR>(out.sh, ad.m.sh, ad.v.sh, g0, cnt, sR, 11, sSH, sUpd, ad.lr_rest, ad.lr_dc, ad);
    }

    if (MODE == 0 && pose_part) {
        __shared__ float red[6][kThreads / 32];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int k = 0; k < 6; k++) {
            float v = pose[k];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
            if (lane == 0) red[k][w] = v;
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            float v = 0.0f;
            for (int ww = 0; ww < kThreads / 32; ww++) v += red[threadIdx.x][ww];
            pose_part[blockIdx.x * 6 + threadIdx.x] = v;
        }
    }
}

struct Jac6 {
    float m[36];
};

__global__ void k_pose_reduce(const float* __restrict__ part, int npart, Jac6 J, float* __restrict__ out6)
{
    // one warp per component, fixed summation order; then J^T g
    __shared__ double gsum[6];
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k < 6) {
        double acc = 0.0;
        for (int i = lane; i < npart; i += 32) acc += part[i * 6 + k];
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
        if (lane == 0) gsum[k] = acc;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double o = 0.0;
        for (int i = 0; i < 6; i++) o += (double)J.m[i * 6 + threadIdx.x] * gsum[i];
        out6[threadIdx.x] = (float)o;
    }
}

template <int MODE>
gl_status launch(View& v, const GParams& p, GMut o, const AdamArgs& a, float* pose_part, cudaStream_t s)
{
    if (p.n == 0) return GL_OK;
    const unsigned grid = (unsigned)((p.n + kThreads - 1) / kThreads);
    PhaseScope ps(v.prof, PH_PARAMS, s);
    count_launches(1);
#define GL_PB(D_)                                                                                         \
    {                                                                                                     \
        GL_TRY(ensure_smem_limit(reinterpret_cast<const void*>(&k_params_bwd<D_, MODE>),                 \
                                 (int)ParamsSmem<D_>::bytes));                                            \
        k_params_bwd<D_, MODE><<<grid, kThreads, ParamsSmem<D_>::bytes, s>>>(                             \
            p, v.d_desc(), v.V, v.radius.as<int>(), v.g2d.as<float>(), o, a, pose_part);                  \
    }
    switch (p.deg) {
        case 0: GL_PB(0); break;
        case 1: GL_PB(1); break;
        case 2: GL_PB(2); break;
        case 3: GL_PB(3); break;
        default: set_error("sh_degree must be 0..3"); return GL_ERR_INVALID;
    }
#undef GL_PB
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

}  // namespace

int pose_partials_needed(int64_t n) { return (int)std::max<int64_t>(1, (n + kThreads - 1) / kThreads); }

gl_status params_backward(View& v, const GParams& p, GMut grad, float* pose_part, int npart, cudaStream_t s)
{
    (void)npart;
    AdamArgs a{};
    return launch<0>(v, p, grad, a, pose_part, s);
}

gl_status params_adam(View& v, const GParams& p, GMut upd, const AdamArgs& a, cudaStream_t s)
{
    return launch<1>(v, p, upd, a, nullptr, s);
}

gl_status pose_reduce(const float* part, int npart, const float jac[36], float* out6, cudaStream_t s)
{
    Jac6 J;
    for (int i = 0; i < 36; i++) J.m[i] = jac[i];
    k_pose_reduce<<<1, 192, 0, s>>>(part, npart, J, out6);
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

}  // namespace gl
