// gl_raster.cu -- per-tile front-to-back compositing (Eq. 4-7) and its adjoint.
//
// Forward: one CTA per screen tile; the tile's depth-sorted Gaussians are
// staged batch by batch into shared memory (gathered through the sorted
// instance list) and every thread blends its pixel(s) front to back until the
// transmittance would fall below 1e-4.  Per pixel it keeps the final
// transmittance and the position of the last blended Gaussian, so the
// backward recomputes T by division instead of storing it per pair.
//
// Backward: the same tiles walked back to front.  Each pixel produces ten
// per-Gaussian partial sums (colour 3, dL/dpower moments 6, depth 1); a warp
// folds its 32 pixels with a transposed butterfly (16 shuffles for 16 slots),
// warps are summed in a fixed order in shared memory, and the result is
// written once per (Gaussian, tile) instance -- no atomics, so the gradients
// are deterministic.
#include "gl_internal.h"

namespace gl {

namespace {

template <int TS>
struct RCfg {
    static constexpr int NT = (TS * TS < 256) ? TS * TS : 256;
    static constexpr int PPT = TS * TS / NT;
    static constexpr int NW = NT / 32 > 0 ? NT / 32 : 1;
};

template <int TS>
__global__ void __launch_bounds__(RCfg<TS>::NT)
k_raster_fwd(const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ sinst,
             const uint32_t* __restrict__ owner, const float4* __restrict__ rec0,
             const float4* __restrict__ rec1, const float4* __restrict__ rec2, int W, int H, int TX,
             float* __restrict__ out_rgb, float* __restrict__ out_depth, float* __restrict__ out_opac,
             float* __restrict__ Tfin, uint32_t* __restrict__ ncon)
{
    constexpr int NT = RCfg<TS>::NT, PPT = RCfg<TS>::PPT;
    __shared__ float4 s0[NT], s1[NT], s2[NT];
    const int tid = threadIdx.x;
    const int tile = blockIdx.x, tx = tile % TX, ty = tile / TX;
    const uint32_t rs = ranges[2 * tile], re = ranges[2 * tile + 1];
    float px[PPT], py[PPT], T[PPT], C0[PPT], C1[PPT], C2[PPT], Dd[PPT], Oo[PPT];
    uint32_t last[PPT];
    bool done[PPT], inside[PPT];
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int local = tid + k * NT;
        const int x = tx * TS + local % TS, y = ty * TS + local / TS;
        px[k] = (float)x; py[k] = (float)y;
        inside[k] = x < W && y < H;
        done[k] = !inside[k];
        T[k] = 1.0f; C0[k] = C1[k] = C2[k] = Dd[k] = Oo[k] = 0.0f;
        last[k] = 0;
    }
    for (uint32_t base = rs; base < re; base += NT) {
        bool mine = true;
#pragma unroll
        for (int k = 0; k < PPT; k++) mine = mine && done[k];
        if (__syncthreads_and(mine)) break;
        const uint32_t i = base + tid;
        if (i < re) {
            const uint32_t g = owner[sinst[i]];
            s0[tid] = rec0[g];
            s1[tid] = rec1[g];
            s2[tid] = rec2[g];
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)NT, re - base);
        for (int j = 0; j < cnt; j++) {
            const float4 a = s0[j], b = s1[j];
            bool alldone = true;
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                if (done[k]) continue;
                alldone = false;
                float dx, dy, alpha, G;
                bool capped;
                if (!pair_alpha(a, b, px[k], py[k], dx, dy, alpha, G, capped)) continue;
                const float tT = __fmul_rn(T[k], __fsub_rn(1.0f, alpha));
                if (tT < kTransMin) { done[k] = true; continue; }
                const float w = alpha * T[k];
                const float4 c = s2[j];
                C0[k] += c.x * w; C1[k] += c.y * w; C2[k] += c.z * w;
                Dd[k] += a.z * w; Oo[k] += w;
                T[k] = tT;
                last[k] = base + j - rs + 1;
            }
            if (alldone) break;
        }
    }
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        if (!inside[k]) continue;
        const size_t p = (size_t)py[k] * W + (size_t)px[k];
        out_rgb[3 * p] = C0[k]; out_rgb[3 * p + 1] = C1[k]; out_rgb[3 * p + 2] = C2[k];
        if (out_depth) out_depth[p] = Dd[k];
        if (out_opac) out_opac[p] = Oo[k];
        Tfin[p] = T[k];
        ncon[p] = last[k];
    }
}

// Sum 16 per-lane values over the warp.  On return lane l holds the total of
// value (l >> 1): each butterfly level halves the slots a lane keeps.
__device__ __forceinline__ float warp_transpose_reduce16(float (&v)[16])
{
    const unsigned lane = threadIdx.x & 31u;
    {
        const bool up = lane & 16u;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            float send = up ? v[k] : v[k + 8];
            float keep = up ? v[k + 8] : v[k];
            v[k] = keep + __shfl_xor_sync(kFull, send, 16);
        }
    }
    {
        const bool up = lane & 8u;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            float send = up ? v[k] : v[k + 4];
            float keep = up ? v[k + 4] : v[k];
            v[k] = keep + __shfl_xor_sync(kFull, send, 8);
        }
    }
    {
        const bool up = lane & 4u;
#pragma unroll
        for (int k = 0; k < 2; k++) {
            float send = up ? v[k] : v[k + 2];
            float keep = up ? v[k + 2] : v[k];
            v[k] = keep + __shfl_xor_sync(kFull, send, 4);
        }
    }
    {
        const bool up = lane & 2u;
        float send = up ? v[0] : v[1];
        float keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(kFull, send, 2);
    }
    return v[0] + __shfl_xor_sync(kFull, v[0], 1);
}

constexpr int kNG = 10;   // per-instance gradient slots
constexpr int kSub = 32;  // Gaussians per flush of the warp partials

template <int TS, bool EXTRA>
__global__ void __launch_bounds__(RCfg<TS>::NT)
k_raster_bwd(const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ sinst,
             const uint32_t* __restrict__ owner, const float4* __restrict__ rec0,
             const float4* __restrict__ rec1, const float4* __restrict__ rec2, int W, int H, int TX,
             const float* __restrict__ Tfin, const uint32_t* __restrict__ ncon,
             const float* __restrict__ dL_drgb, const float* __restrict__ dL_ddepth,
             const float* __restrict__ dL_dopac, float* __restrict__ igrad)
{
    constexpr int NT = RCfg<TS>::NT, PPT = RCfg<TS>::PPT, NW = RCfg<TS>::NW;
    __shared__ float4 s0[NT], s1[NT], s2[NT];
    __shared__ uint32_t sd[NT];
    __shared__ float part[NW][kSub][kNG];
    __shared__ uint32_t s_max;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int tile = blockIdx.x, tx = tile % TX, ty = tile / TX;
    const uint32_t rs = ranges[2 * tile], re = ranges[2 * tile + 1];

    float px[PPT], py[PPT], T[PPT], R0[PPT], R1[PPT], R2[PPT], RD[PPT], RO[PPT];
    float g0[PPT], g1[PPT], g2[PPT], gD[PPT], gO[PPT];
    uint32_t last[PPT];
    if (tid == 0) s_max = 0;
    __syncthreads();
    uint32_t mymax = 0;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int local = tid + k * NT;
        const int x = tx * TS + local % TS, y = ty * TS + local / TS;
        px[k] = (float)x; py[k] = (float)y;
        R0[k] = R1[k] = R2[k] = RD[k] = RO[k] = 0.0f;
        g0[k] = g1[k] = g2[k] = gD[k] = gO[k] = 0.0f;
        T[k] = 1.0f;
        last[k] = 0;
        if (x < W && y < H) {
            const size_t p = (size_t)y * W + x;
            T[k] = Tfin[p];
            last[k] = ncon[p];
            g0[k] = dL_drgb[3 * p]; g1[k] = dL_drgb[3 * p + 1]; g2[k] = dL_drgb[3 * p + 2];
            if (EXTRA) {
                gD[k] = dL_ddepth ? dL_ddepth[p] : 0.0f;
                gO[k] = dL_dopac ? dL_dopac[p] : 0.0f;
            }
        }
        mymax = max(mymax, last[k]);
    }
    atomicMax(&s_max, mymax);
    __syncthreads();
    const uint32_t end = rs + s_max;
    // instances no pixel reached get zero gradients
    for (uint32_t i = end + tid; i < re; i += NT) {
        float* o = igrad + (size_t)sinst[i] * kNG;
#pragma unroll
        for (int q = 0; q < kNG; q++) o[q] = 0.0f;
    }
    for (int64_t bend = end; bend > (int64_t)rs; bend -= NT) {
        const int64_t bstart = bend - NT > (int64_t)rs ? bend - NT : (int64_t)rs;
        const int cnt = (int)(bend - bstart);
        __syncthreads();
        if (tid < cnt) {
            const uint32_t d = sinst[bstart + tid];
            const uint32_t g = owner[d];
            sd[tid] = d;
            s0[tid] = rec0[g];
            s1[tid] = rec1[g];
            s2[tid] = rec2[g];
        }
        __syncthreads();
        for (int sub_end = cnt; sub_end > 0; sub_end -= kSub) {
            const int sub_start = sub_end - kSub > 0 ? sub_end - kSub : 0;
            for (int j = sub_end - 1; j >= sub_start; j--) {
                const float4 a = s0[j], b = s1[j], c = s2[j];
                const uint32_t pos = (uint32_t)(bstart + j) - rs;
                float v[16];
#pragma unroll
                for (int q = 0; q < 16; q++) v[q] = 0.0f;
                bool any = false;
#pragma unroll
                for (int k = 0; k < PPT; k++) {
                    if (pos >= last[k]) continue;
                    float dx, dy, alpha, G;
                    bool capped;
                    if (!pair_alpha(a, b, px[k], py[k], dx, dy, alpha, G, capped)) continue;
                    T[k] = __fdiv_rn(T[k], __fsub_rn(1.0f, alpha));
                    const float wgt = alpha * T[k];
                    float ga = g0[k] * (c.x - R0[k]) + g1[k] * (c.y - R1[k]) + g2[k] * (c.z - R2[k]);
                    if (EXTRA) ga += gD[k] * (a.z - RD[k]) + gO[k] * (1.0f - RO[k]);
                    ga *= T[k];
                    const float om = 1.0f - alpha;
                    R0[k] = alpha * c.x + om * R0[k];
                    R1[k] = alpha * c.y + om * R1[k];
                    R2[k] = alpha * c.z + om * R2[k];
                    if (EXTRA) {
                        RD[k] = alpha * a.z + om * RD[k];
                        RO[k] = alpha + om * RO[k];
                    }
                    const float gp = capped ? 0.0f : ga * alpha;
                    v[0] += wgt * g0[k]; v[1] += wgt * g1[k]; v[2] += wgt * g2[k];
                    v[3] += gp;
                    v[4] += gp * dx; v[5] += gp * dy;
                    v[6] += gp * dx * dx; v[7] += gp * dx * dy; v[8] += gp * dy * dy;
                    if (EXTRA) v[9] += wgt * gD[k];
                    any = true;
                }
                const int jj = j - sub_start;
                if (__any_sync(kFull, any)) {
                    const float r = warp_transpose_reduce16(v);
                    if ((lane & 1) == 0 && (lane >> 1) < kNG) part[w][jj][lane >> 1] = r;
                } else if (lane < kNG) {
                    part[w][jj][lane] = 0.0f;
                }
            }
            __syncthreads();
            const int nsub = sub_end - sub_start;
            for (int e = tid; e < nsub * kNG; e += NT) {
                const int jj = e / kNG, q = e % kNG;
                float s = 0.0f;
#pragma unroll
                for (int ww = 0; ww < NW; ww++) s += part[ww][jj][q];
                igrad[(size_t)sd[sub_start + jj] * kNG + q] = s;
            }
            __syncthreads();
        }
    }
}

}  // namespace

gl_status raster_forward(View& v, float* rgb, float* depth, float* opac, cudaStream_t s)
{
    const size_t P = (size_t)v.W * v.H;
    GL_TRY(v.Tfin.reserve(4 * P));
    GL_TRY(v.ncon.reserve(4 * P));
    if (v.ntiles == 0) return GL_OK;
    PhaseScope ps(v.prof, PH_RASTER_FWD, s);
    count_launches(1);
    const uint32_t* own = v.iowner.as<uint32_t>();
#define GL_FWD(TS_)                                                                          \
    k_raster_fwd<TS_><<<v.ntiles, RCfg<TS_>::NT, 0, s>>>(                                    \
        v.ranges.as<uint32_t>(), v.sorted_inst, own, v.rec0.as<float4>(), v.rec1.as<float4>(), \
        v.rec2.as<float4>(), v.W, v.H, v.TX, rgb, depth, opac, v.Tfin.as<float>(),           \
        v.ncon.as<uint32_t>())
    switch (v.Ts) {
        case 8: GL_FWD(8); break;
        case 16: GL_FWD(16); break;
        case 32: GL_FWD(32); break;
        default: set_error("tile_size must be 8, 16 or 32"); return GL_ERR_INVALID;
    }
#undef GL_FWD
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

gl_status raster_backward(View& v, const float* dL_drgb, const float* dL_ddepth,
                          const float* dL_dopac, cudaStream_t s)
{
    if (v.ntiles == 0 || v.I == 0) return GL_OK;
    const bool extra = dL_ddepth != nullptr || dL_dopac != nullptr;
    PhaseScope ps(v.prof, PH_RASTER_BWD, s);
    count_launches(1);
    const uint32_t* own = v.iowner.as<uint32_t>();
#define GL_BWD(TS_, EX_)                                                                      \
    k_raster_bwd<TS_, EX_><<<v.ntiles, RCfg<TS_>::NT, 0, s>>>(                                \
        v.ranges.as<uint32_t>(), v.sorted_inst, own, v.rec0.as<float4>(), v.rec1.as<float4>(),  \
        v.rec2.as<float4>(), v.W, v.H, v.TX, v.Tfin.as<float>(), v.ncon.as<uint32_t>(), dL_drgb, \
        dL_ddepth, dL_dopac, v.igrad.as<float>())
    switch (v.Ts) {
        case 8: if (extra) GL_BWD(8, true); else GL_BWD(8, false); break;
        case 16: if (extra) GL_BWD(16, true); else GL_BWD(16, false); break;
        case 32: if (extra) GL_BWD(32, true); else GL_BWD(32, false); break;
        default: set_error("tile_size must be 8, 16 or 32"); return GL_ERR_INVALID;
    }
#undef GL_BWD
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

}  // namespace gl
