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

constexpr int kPG = 32;   // Gaussians per CTA: one warp, one Gaussian per lane
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
    // the backward's geometry divides by the hardware's approximate
    // reciprocal and exponentiates by its approximate exponential (a few ulp;
    // the gradients' tolerance is 1e-3): no divide sequences on the chain
    G.iz = __fdividef(1.0f, G.z);
    for (int i = 0; i < 3; i++) G.s[i] = __expf(ls[i]);
    float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    G.qnorm = sqrtf(qq);
    const float inv = __fdividef(1.0f, G.qnorm);
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
    const float limx = kJacClamp * __fdividef(0.5f * (float)cam.W, cam.fx);
    const float limy = kJacClamp * __fdividef(0.5f * (float)cam.H, cam.fy);
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
    const float idet = __fdividef(1.0f, G.a * G.c - G.b * G.b);
    G.A = G.c * idet;
    G.B = -G.b * idet;
    G.C = G.a * idet;
    G.o = __fdividef(1.0f, 1.0f + __expf(-logit));
    const float cw0 = -(R[0] * cam.t[0] + R[3] * cam.t[1] + R[6] * cam.t[2]);
    const float cw1 = -(R[1] * cam.t[0] + R[4] * cam.t[1] + R[7] * cam.t[2]);
    const float cw2 = -(R[2] * cam.t[0] + R[5] * cam.t[1] + R[8] * cam.t[2]);
    const float d0 = mu[0] - cw0, d1 = mu[1] - cw1, d2 = mu[2] - cw2;
    const float dd2 = d0 * d0 + d1 * d1 + d2 * d2;
    G.dnorm = sqrtf(dd2);
    const float idn = __fdividef(1.0f, G.dnorm);
    G.dir[0] = d0 * idn; G.dir[1] = d1 * idn; G.dir[2] = d2 * idn;
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

// ---------------------------------------------------------------------------
// Bulk copies global -> shared memory (the copy engine behind TMA, untiled
// form), completing on an mbarrier; each span starts and ends on 16 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return done != 0;
}

// Polls of a staging barrier before the kernel gives up (each poll may
// suspend the thread for a while): far beyond any real copy time.
constexpr int kStageSpin = 1 << 22;

// Hint the L2 to fetch [p, p + bytes) (its 16-byte aligned part) with one
// bulk prefetch; nothing waits for it.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes)
{
    const uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
    const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
    if (e > a) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(e - a)) : "memory");
}

// Staged rows of a block of kPG Gaussians: each parameter array's span,
// dense as in global memory, then the gradient rows at an odd stride
// (against bank conflicts).  Offsets in floats; every span starts on 16
// bytes.
template <int DEG, int MODE>
struct PStage {
    static constexpr int KF = (DEG + 1) * (DEG + 1) * 3;
    static constexpr int ROW = 11 + KF;                      // floats of one Gaussian's parameters
    static constexpr int MU = 0, LS = 3 * kPG, Q = 6 * kPG, LG = 10 * kPG, SH = 11 * kPG;
    static constexpr int SET = ROW * kPG;                    // the parameter rows
    static constexpr int NSET = 1;
    static constexpr int NR = ROW % 2 ? ROW : ROW + 1;
    static constexpr int GR = NSET * SET;                    // gradient rows
    static constexpr int FLOATS = GR + NR * kPG;
    static_assert(SET % 4 == 0 && LG % 4 == 0 && SH % 4 == 0, "16-byte spans");
};

// Copy one array's span [g0, g0 + cnt) rows of WIDTH floats into shared
// memory: a bulk copy for a whole block (cnt = kPG), lane-strided loads for
// the last, partial one.
template <int WIDTH>
__device__ __forceinline__ void stage_span(const float* __restrict__ src, int64_t g0, int cnt, float* dst,
                                           uint64_t* bar, int lane)
{
    const float* s0 = src + (size_t)g0 * WIDTH;
    if (cnt == kPG) {
        if (lane == 0) bulk_g2s(dst, s0, (uint32_t)(sizeof(float) * WIDTH * kPG), bar);
    } else {
        for (int e = lane; e < cnt * WIDTH; e += 32) dst[e] = s0[e];
    }
}

// Adam (MODE 1) or the gradient write-out (MODE 0) over one array's span:
// element e of the span is row e / WIDTH, column e % WIDTH; the parameter
// comes from the staged rows, m and v from global memory (already asked of
// the L2), the gradient from the row's gradient (columns from `off`).  Whole
// blocks go by float4 (a float4 may straddle rows; the elements of rows left
// alone are written back unchanged), the partial block element by element.
// Rows whose bit in `upd` is clear are left untouched (FULL: every row of a
// whole block is updated, and no row is tested).  On the SH span (WIDTH > 4)
// the first three columns take lr0 (the DC band), the rest lr.
template <int MODE, int WIDTH, int NR, bool FULL = false>
__device__ __forceinline__ void span_update(float* __restrict__ P, float* __restrict__ Mg, float* __restrict__ Vg,
                                            int64_t g0, int cnt, const float* sP, const float* sR, int off,
                                            uint32_t upd, float lr, float lr0, const AdamArgs& ad, int lane)
{
    const size_t base = (size_t)g0 * WIDTH;
    if (cnt == kPG) {
        constexpr int N4 = WIDTH * kPG / 4;
#pragma unroll 4
        for (int c = lane; c < N4; c += 32) {
            // rows and columns of the four elements: one division, then the
            // column steps by one and wraps into the next row
            const int e0 = 4 * c;
            int rr[4], ww[4];
            rr[0] = e0 / WIDTH;
            ww[0] = e0 - rr[0] * WIDTH;
#pragma unroll
            for (int k = 1; k < 4; k++) {
                const bool wrap = ww[k - 1] + 1 == WIDTH;
                ww[k] = wrap ? 0 : ww[k - 1] + 1;
                rr[k] = rr[k - 1] + (wrap ? 1 : 0);
            }
            const uint32_t rows = FULL ? 1u : (upd >> rr[0]) & ((2u << (rr[3] - rr[0])) - 1u);
            if (!rows) continue;
            float pe[4], me[4], ve[4];
            if (MODE == 1) {
                const float4 pp = reinterpret_cast<const float4*>(sP)[c];
                // moments and parameters are touched once per step: streaming
                // loads and stores leave the L2 to the moments prefetched for
                // the blocks still to come
                const float4 mm = __ldcs(reinterpret_cast<const float4*>(Mg + base) + c);
                const float4 vv = __ldcs(reinterpret_cast<const float4*>(Vg + base) + c);
                pe[0] = pp.x; pe[1] = pp.y; pe[2] = pp.z; pe[3] = pp.w;
                me[0] = mm.x; me[1] = mm.y; me[2] = mm.z; me[3] = mm.w;
                ve[0] = vv.x; ve[1] = vv.y; ve[2] = vv.z; ve[3] = vv.w;
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int r = rr[k], w = ww[k];
                const float g = sR[r * NR + off + w];
                if (MODE == 0) pe[k] = (FULL || ((upd >> r) & 1u)) ? g : 0.0f;
                else if (FULL || ((upd >> r) & 1u)) adam1(pe[k], me[k], ve[k], g, (WIDTH > 4 && w < 3) ? lr0 : lr, ad);
            }
            __stcs(reinterpret_cast<float4*>(P + base) + c, make_float4(pe[0], pe[1], pe[2], pe[3]));
            if (MODE == 1) {
                __stcs(reinterpret_cast<float4*>(Mg + base) + c, make_float4(me[0], me[1], me[2], me[3]));
                __stcs(reinterpret_cast<float4*>(Vg + base) + c, make_float4(ve[0], ve[1], ve[2], ve[3]));
            }
        }
    } else {
        for (int e = lane; e < cnt * WIDTH; e += 32) {
            const int r = e / WIDTH, w = e - r * WIDTH;
            if (!((upd >> r) & 1u)) {
                if (MODE == 0) P[base + e] = 0.0f;
                continue;
            }
            const float g = sR[r * NR + off + w];
            if (MODE == 0) {
                P[base + e] = g;
            } else {
                float pv = sP[e], mv = Mg[base + e], vv = Vg[base + e];
                adam1(pv, mv, vv, g, w < 3 ? lr0 : lr, ad);
                P[base + e] = pv;
                Mg[base + e] = mv;
                Vg[base + e] = vv;
            }
        }
    }
}

// One warp per kPG consecutive Gaussians, 128 registers a thread, so that
// 16 warps share an SM.  The block's visibility comes first (a block with
// nothing visible is skipped by sparse Adam, or written as zero gradients);
// then one lane starts bulk copies of the block's rows of every parameter
// array into shared memory (7.5 KB in flight per block whatever the thread
// count) and bulk L2 prefetches of its Adam moments; each lane chains its
// Gaussian's screen-space gradients back to the parameters (and the pose),
// and the warp applies Adam -- or writes the gradients -- array by array with
// float4 accesses.  Parameters and moments are read once and written once,
// and sparse Adam touches no moment of a block it skips.
template <int DEG, int MODE>
__global__ void __launch_bounds__(32, 16)
k_params_bwd(GParams p, const ViewDesc* __restrict__ views, int V, const int* __restrict__ radius,
             const float* __restrict__ g2d, GMut out, AdamArgs ad, float* __restrict__ pose_part,
             unsigned long long* __restrict__ err)
{
    using ST = PStage<DEG, MODE>;
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int KF = ST::KF;
    constexpr int NR = ST::NR;
    if (MODE == 1) {
        // a step whose binning overflowed its buffers updates nothing (it is re-run)
        if (ad.abort && ad.abort[1]) return;
        if (ad.bc) { ad.ibc1 = ad.bc[0]; ad.isbc2 = ad.bc[1]; }
    }
    __shared__ __align__(16) float smf[ST::FLOATS];
    __shared__ uint64_t bar;
    const int lane = threadIdx.x;
    const int64_t g0 = blockIdx.x * (int64_t)kPG;
    const int cnt = (int)min((int64_t)kPG, p.n - g0);
    const int64_t g = g0 + lane;
    const bool valid = lane < cnt;
    bool vis = false;
    for (int vw = 0; vw < V && valid; vw++) vis = vis || radius[(size_t)vw * p.n + g] > 0;
    const uint32_t vmask = __ballot_sync(kFull, vis);
    const uint32_t vrows = __ballot_sync(kFull, valid);
    const uint32_t upd = MODE == 0 ? vrows : (ad.sparse ? vmask : vrows);
    if (MODE == 1 && upd == 0) return;

    float* sMu = smf + ST::MU;
    float* sLs = smf + ST::LS;
    float* sQ = smf + ST::Q;
    float* sLg = smf + ST::LG;
    float* sSH = smf + ST::SH;
    float* sR = smf + ST::GR;
    float pose[6] = {0, 0, 0, 0, 0, 0};
    if (vmask) {
        const bool bulk = cnt == kPG;
        if (bulk && lane == 0) {
            mbar_init(&bar, 1);
            mbar_expect_tx(&bar, (uint32_t)(sizeof(float) * ST::SET * ST::NSET));
        }
        __syncwarp();
        stage_span<3>(p.means, g0, cnt, sMu, &bar, lane);
        stage_span<3>(p.log_scales, g0, cnt, sLs, &bar, lane);
        stage_span<4>(p.quats, g0, cnt, sQ, &bar, lane);
        stage_span<1>(p.logits, g0, cnt, sLg, &bar, lane);
        stage_span<KF>(p.sh, g0, cnt, sSH, &bar, lane);
        if (MODE == 1 && lane == 0) {
            // the moments head for the L2 while the geometry is recomputed
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
        if (bulk) {
            // bounded wait; on giving up, raise the flag and wait once more
            // (again bounded) for the copies still landing in this block's
            // shared memory before leaving
            int spins = 0;
            bool ok = mbar_try_wait(&bar, 0);
            while (!ok && ++spins < kStageSpin) ok = mbar_try_wait(&bar, 0);
            if (!__all_sync(kFull, ok)) {
                if (lane == 0) atomicOr(err, 2ull);
                for (int k = 0; k < kStageSpin && !ok; k++) ok = mbar_try_wait(&bar, 0);
                return;
            }
        }
        __syncwarp();

        bool first = true;
        float gm[3] = {0, 0, 0}, gl3[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, glg = 0.0f;
        float* dsh = sR + lane * NR + 11;   // this Gaussian's SH gradient, summed over its views in place

    // every view the Gaussian is visible in contributes (window steps sum them)
    for (int vw = 0; vw < V && valid; vw++) {
    const int64_t tv = (int64_t)vw * p.n + g;
    if (radius[tv] <= 0) continue;
    const Cam cam = views[vw].cam;
    float grgb[3] = {0, 0, 0};
    {
        float Y[16];
        const int r = lane;
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
        const float dz = s[9];

        // opacity: alpha = o exp(power), so dL/do = s[3] / o and
        // dL/dlogit = dL/do o (1 - o) = s[3] (1 - o), with no division
        glg += s[3] * (1.0f - G.o);

        // colour -> SH and view direction (clamped channels pass no gradient)
        sh_eval<DEG>(G.dir[0], G.dir[1], G.dir[2], Y);
        const float* sh = sSH + lane * KF;
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
        for (int j = 0; j < 3; j++) gdu[j] = __fdividef(gdir[j] - G.dir[j] * dd, G.dnorm);
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
            for (int i = 0; i < 4; i++) gq[i] += __fdividef(gn[i] - G.qn[i] * qd, G.qnorm);
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
        float* row = sR + lane * NR;
        row[0] = gm[0]; row[1] = gm[1]; row[2] = gm[2];
        row[3] = gl3[0]; row[4] = gl3[1]; row[5] = gl3[2];
        row[6] = gq[0]; row[7] = gq[1]; row[8] = gq[2]; row[9] = gq[3];
        row[10] = glg;
        __syncwarp();
    } else {
        // nothing visible: zero gradients (MODE 0, and dense Adam, which
        // still moves every row on its moments; sparse Adam returned above)
        for (int e = lane; e < kPG * NR; e += 32) sR[e] = 0.0f;
        __syncwarp();
    }
    if (MODE == 1 && !vmask) {
        // dense Adam on a block nothing sees: its parameter rows, staged plainly
        const float* srcs[5] = {p.means, p.log_scales, p.quats, p.logits, p.sh};
        float* dsts[5] = {sMu, sLs, sQ, sLg, sSH};
        const int widths[5] = {3, 3, 4, 1, KF};
        for (int a = 0; a < 5; a++) {
            const float* s0 = srcs[a] + (size_t)g0 * widths[a];
            for (int e = lane; e < cnt * widths[a]; e += 32) dsts[a][e] = s0[e];
        }
        __syncwarp();
    }
    // every row of a whole block updated: the spans skip the row tests
    if (upd == kFull && cnt == kPG) {
        span_update<MODE, 3, NR, true>(out.means, ad.m.means, ad.v.means, g0, cnt, sMu, sR, 0, upd, ad.lr_pos,
                                       ad.lr_pos, ad, lane);
        span_update<MODE, 3, NR, true>(out.log_scales, ad.m.log_scales, ad.v.log_scales, g0, cnt, sLs, sR, 3, upd,
                                       ad.lr_scale, ad.lr_scale, ad, lane);
        span_update<MODE, 4, NR, true>(out.quats, ad.m.quats, ad.v.quats, g0, cnt, sQ, sR, 6, upd, ad.lr_rot,
                                       ad.lr_rot, ad, lane);
        span_update<MODE, 1, NR, true>(out.logits, ad.m.logits, ad.v.logits, g0, cnt, sLg, sR, 10, upd, ad.lr_op,
                                       ad.lr_op, ad, lane);
        span_update<MODE, KF, NR, true>(out.sh, ad.m.sh, ad.v.sh, g0, cnt, sSH, sR, 11, upd, ad.lr_rest, ad.lr_dc,
                                        ad, lane);
    } else {
        span_update<MODE, 3, NR>(out.means, ad.m.means, ad.v.means, g0, cnt, sMu, sR, 0, upd, ad.lr_pos, ad.lr_pos,
                                 ad, lane);
        span_update<MODE, 3, NR>(out.log_scales, ad.m.log_scales, ad.v.log_scales, g0, cnt, sLs, sR, 3, upd,
                                 ad.lr_scale, ad.lr_scale, ad, lane);
        span_update<MODE, 4, NR>(out.quats, ad.m.quats, ad.v.quats, g0, cnt, sQ, sR, 6, upd, ad.lr_rot, ad.lr_rot,
                                 ad, lane);
        span_update<MODE, 1, NR>(out.logits, ad.m.logits, ad.v.logits, g0, cnt, sLg, sR, 10, upd, ad.lr_op,
                                 ad.lr_op, ad, lane);
        span_update<MODE, KF, NR>(out.sh, ad.m.sh, ad.v.sh, g0, cnt, sSH, sR, 11, upd, ad.lr_rest, ad.lr_dc, ad,
                                  lane);
    }

    if (MODE == 0 && pose_part) {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            float v = pose[k];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
            if (lane == 0) pose_part[blockIdx.x * 6 + k] = v;
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
        // partials lane, lane + 32, ... in that order, 8 loads in flight
        double acc = 0.0;
        for (int i0 = lane; i0 < npart; i0 += 256) {
            float x[8];
#pragma unroll
            for (int b = 0; b < 8; b++) x[b] = i0 + 32 * b < npart ? part[(size_t)(i0 + 32 * b) * 6 + k] : 0.0f;
#pragma unroll
            for (int b = 0; b < 8; b++)
                if (i0 + 32 * b < npart) acc += x[b];
        }
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
    const unsigned grid = (unsigned)((p.n + kPG - 1) / kPG);
    PhaseScope ps(v.prof, PH_PARAMS, s);
    count_launches(1);
    unsigned long long* err = reinterpret_cast<unsigned long long*>(v.count.as<uint64_t>() + 8);
#define GL_PB(D_)                                                                                      \
    k_params_bwd<D_, MODE><<<grid, kPG, 0, s>>>(p, v.d_desc(), v.V, v.radius.as<int>(), v.g2d.as<float>(), o, a, \
                                                pose_part, err);
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

int pose_partials_needed(int64_t n) { return (int)std::max<int64_t>(1, (n + kPG - 1) / kPG); }

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
