// gl_raster.cu -- front-to-back compositing (Eq. 4-7) and its adjoint.
//
// Work unit: one warp per (screen tile, 8x4 pixel block).  Binning is done
// per tile (TS x TS), but every 8x4 block of a tile is rendered by its own
// warp, independently: a heavy tile is spread over TS*TS/32 warps instead of
// being the critical path of one CTA.  Units are launched heaviest tile first.
//
// Records are permuted into sorted-instance order after binning, so a tile's
// Gaussians are contiguous: each lane loads one Gaussian per batch of 32
// (prefetched one batch ahead), the warp ballots which Gaussians' alpha boxes
// touch its pixel block, compacts those hits in shared memory in depth order
// and evaluates only them.  A Gaussian outside the block's box fails the
// alpha test at every pixel of the block, so skipping it changes no result.
//
// Forward: per pixel, blend until the transmittance would fall below 1e-4;
// keep the final transmittance and the position (in the tile's list) of the
// last blended Gaussian, so the backward recomputes T by division.
// Backward: the same units walked back to front; per hit, the warp folds its
// 32 pixels' ten partial sums (colour 3, dL/dpower moments 6, depth 1) with a
// transposed butterfly and ten lanes add them to the Gaussian's accumulator.
#include "gl_internal.h"

namespace gl {

namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kNG = 10;   // screen-space gradient slots per Gaussian

struct Unit {
    int x0, y0;            // absolute pixel origin of the 8x4 block in its view
    int W, H;              // the view's image size
    long long pix_base;    // the view's first pixel in the concatenated images
    uint32_t rs, re;       // the tile's list
};

__device__ __forceinline__ void unit_of(int u, int TS, const ViewDesc* __restrict__ views, int V,
                                        const uint32_t* __restrict__ order,
                                        const uint32_t* __restrict__ ranges, Unit& U)
{
    const int wb_per_tile = TS * TS / 32, bpr = TS / 8;
    const int tile = (int)order[u / wb_per_tile], wb = u % wb_per_tile;
    const int v = view_of_tile(views, V, tile);
    const ViewDesc& d = views[v];
    const int lt = tile - d.tile_base;
    U.x0 = (lt % d.TX) * TS + (wb % bpr) * 8;
    U.y0 = (lt / d.TX) * TS + (wb / bpr) * 4;
    U.W = d.cam.W;
    U.H = d.cam.H;
    U.pix_base = d.pix_base;
    U.rs = ranges[2 * tile];
    U.re = ranges[2 * tile + 1];
}

__device__ __forceinline__ bool box_hit(const float4 box, float bx0, float bx1, float by0, float by1)
{
    return !(box.y < bx0 || box.x > bx1 || box.w < by0 || box.z > by1);
}

__global__ void __launch_bounds__(32 * kWarpsPerBlock)
k_raster_fwd(int nunits, int TS, const uint32_t* __restrict__ order, const uint32_t* __restrict__ ranges,
             const float4* __restrict__ s0g, const float4* __restrict__ s1g, const float4* __restrict__ s2g,
             const float4* __restrict__ s3g, const ViewDesc* __restrict__ views, int V,
             float* __restrict__ out_rgb,
             float* __restrict__ out_depth, float* __restrict__ out_opac, float* __restrict__ Tfin,
             uint32_t* __restrict__ ncon)
{
    __shared__ float4 sr0[kWarpsPerBlock][32], sr1[kWarpsPerBlock][32], sr2[kWarpsPerBlock][32];
    __shared__ uint32_t spos[kWarpsPerBlock][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int u = blockIdx.x * kWarpsPerBlock + w;
    if (u >= nunits) return;
    Unit U;
    unit_of(u, TS, views, V, order, ranges, U);
    const int x = U.x0 + (lane & 7), y = U.y0 + (lane >> 3);
    const bool inside = x < U.W && y < U.H;
    const float px = (float)x, py = (float)y;
    const float bx0 = (float)U.x0, bx1 = (float)(U.x0 + 7), by0 = (float)U.y0, by1 = (float)(U.y0 + 3);
    const unsigned lt = (1u << lane) - 1u;
    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f, Dd = 0.f, Oo = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    // prefetch of the first batch
    float4 n0, n1, n2, n3;
    {
        const uint32_t i = U.rs + lane;
        if (i < U.re) { n0 = s0g[i]; n1 = s1g[i]; n2 = s2g[i]; n3 = s3g[i]; }
    }
    for (uint32_t base = U.rs; base < U.re; base += 32) {
        if (__all_sync(kFull, done)) break;
        const float4 c0 = n0, c1 = n1, c2 = n2, c3 = n3;
        const uint32_t i = base + lane;
        const bool valid = i < U.re;
        const uint32_t ni = i + 32;
        if (ni < U.re) { n0 = s0g[ni]; n1 = s1g[ni]; n2 = s2g[ni]; n3 = s3g[ni]; }
        const bool hit = valid && box_hit(c3, bx0, bx1, by0, by1);
        const unsigned mask = __ballot_sync(kFull, hit);
        if (hit) {
            const int k = __popc(mask & lt);
            sr0[w][k] = c0; sr1[w][k] = c1; sr2[w][k] = c2;
            spos[w][k] = i - U.rs;
        }
        __syncwarp();
        const int nh = __popc(mask);
        for (int k = 0; k < nh; k++) {
            if (done) break;
            float dx, dy, alpha;
            bool capped;
            const float4 a = sr0[w][k], b = sr1[w][k];
            if (!pair_eval(a, b, px, py, dx, dy, alpha, capped)) continue;
            const float tT = __fmul_rn(T, __fsub_rn(1.0f, alpha));
            if (tT < kTransMin) { done = true; break; }
            const float wgt = alpha * T;
            const float4 c = sr2[w][k];
            C0 += c.x * wgt; C1 += c.y * wgt; C2 += c.z * wgt;
            Dd += b.z * wgt; Oo += wgt;
            T = tT;
            last = spos[w][k] + 1;
        }
        __syncwarp();
    }
    if (!inside) return;
    const size_t p = (size_t)U.pix_base + (size_t)y * U.W + x;
    out_rgb[3 * p] = C0; out_rgb[3 * p + 1] = C1; out_rgb[3 * p + 2] = C2;
    if (out_depth) out_depth[p] = Dd;
    if (out_opac) out_opac[p] = Oo;
    Tfin[p] = T;
    ncon[p] = last;
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

template <bool EXTRA>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
k_raster_bwd(int nunits, int TS, const uint32_t* __restrict__ order, const uint32_t* __restrict__ ranges,
             const float4* __restrict__ s0g, const float4* __restrict__ s1g, const float4* __restrict__ s2g,
             const float4* __restrict__ s3g, const uint32_t* __restrict__ sgid,
             const ViewDesc* __restrict__ views, int V,
             const float* __restrict__ Tfin, const uint32_t* __restrict__ ncon,
             const float* __restrict__ dL_drgb, const float* __restrict__ dL_ddepth,
             const float* __restrict__ dL_dopac, float* __restrict__ g2d)
{
    __shared__ float4 sr0[kWarpsPerBlock][32], sr1[kWarpsPerBlock][32], sr2[kWarpsPerBlock][32];
    __shared__ uint32_t spos[kWarpsPerBlock][32], sg[kWarpsPerBlock][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int u = blockIdx.x * kWarpsPerBlock + w;
    if (u >= nunits) return;
    Unit U;
    unit_of(u, TS, views, V, order, ranges, U);
    const int x = U.x0 + (lane & 7), y = U.y0 + (lane >> 3);
    const bool inside = x < U.W && y < U.H;
    const float px = (float)x, py = (float)y;
    const float bx0 = (float)U.x0, bx1 = (float)(U.x0 + 7), by0 = (float)U.y0, by1 = (float)(U.y0 + 3);
    const unsigned lt = (1u << lane) - 1u;
    float T = 1.0f, R0 = 0.f, R1 = 0.f, R2 = 0.f, RD = 0.f, RO = 0.f;
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, gD = 0.f, gO = 0.f;
    uint32_t last = 0;
    if (inside) {
        const size_t p = (size_t)U.pix_base + (size_t)y * U.W + x;
        T = Tfin[p];
        last = ncon[p];
        g0 = dL_drgb[3 * p]; g1 = dL_drgb[3 * p + 1]; g2 = dL_drgb[3 * p + 2];
        if (EXTRA) {
            gD = dL_ddepth ? dL_ddepth[p] : 0.0f;
            gO = dL_dopac ? dL_dopac[p] : 0.0f;
        }
    }
    uint32_t wmax = last;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wmax = max(wmax, __shfl_xor_sync(kFull, wmax, off));
    const uint32_t end = U.rs + wmax;   // positions at or beyond this reach no pixel of the block
    if (end == U.rs) return;
    // batches from the back: [bstart, bstart + 32) with bstart = end - 32 k, clipped at rs
    int64_t bstart = (int64_t)end - 32;
    float4 n0, n1, n2, n3;
    uint32_t ng = 0;
    {
        const int64_t i = bstart + lane;
        if (i >= (int64_t)U.rs) { n0 = s0g[i]; n1 = s1g[i]; n2 = s2g[i]; n3 = s3g[i]; ng = sgid[i]; }
    }
    for (; bstart + 32 > (int64_t)U.rs; bstart -= 32) {
        const float4 c0 = n0, c1 = n1, c2 = n2, c3 = n3;
        const uint32_t cg = ng;
        const int64_t i = bstart + lane;
        const bool valid = i >= (int64_t)U.rs;
        const int64_t ni = i - 32;
        if (ni >= (int64_t)U.rs) { n0 = s0g[ni]; n1 = s1g[ni]; n2 = s2g[ni]; n3 = s3g[ni]; ng = sgid[ni]; }
        const bool hit = valid && box_hit(c3, bx0, bx1, by0, by1);
        const unsigned mask = __ballot_sync(kFull, hit);
        if (hit) {
            const int k = __popc(mask & lt);
            sr0[w][k] = c0; sr1[w][k] = c1; sr2[w][k] = c2;
            spos[w][k] = (uint32_t)(i - U.rs);
            sg[w][k] = cg;
        }
        __syncwarp();
        const int nh = __popc(mask);
        for (int k = nh - 1; k >= 0; k--) {
            const float4 a = sr0[w][k], b = sr1[w][k], c = sr2[w][k];
            float v[16];
#pragma unroll
            for (int q = 0; q < 16; q++) v[q] = 0.0f;
            bool any = false;
            float dx, dy, alpha;
            bool capped;
            if (spos[w][k] < last && pair_eval(a, b, px, py, dx, dy, alpha, capped)) {
                const float om = 1.0f - alpha;
                T = __fdividef(T, om);
                const float wgt = alpha * T;
                float ga = g0 * (c.x - R0) + g1 * (c.y - R1) + g2 * (c.z - R2);
                if (EXTRA) ga += gD * (b.z - RD) + gO * (1.0f - RO);
                ga *= T;
                R0 = alpha * c.x + om * R0;
                R1 = alpha * c.y + om * R1;
                R2 = alpha * c.z + om * R2;
                if (EXTRA) {
                    RD = alpha * b.z + om * RD;
                    RO = alpha + om * RO;
                }
                const float gp = capped ? 0.0f : ga * alpha;
                v[0] = wgt * g0; v[1] = wgt * g1; v[2] = wgt * g2;
                v[3] = gp;
                v[4] = gp * dx; v[5] = gp * dy;
                v[6] = gp * dx * dx; v[7] = gp * dx * dy; v[8] = gp * dy * dy;
                if (EXTRA) v[9] = wgt * gD;
                any = true;
            }
            if (__any_sync(kFull, any)) {
                const float r = warp_transpose_reduce16(v);
                const int q = lane >> 1;
                if ((lane & 1) == 0 && q < (EXTRA ? kNG : kNG - 1))
                    atomicAdd(g2d + (size_t)sg[w][k] * kNG + q, r);
            }
        }
        __syncwarp();
    }
}

// Records in sorted-instance order (and the owning Gaussian of each).
__global__ void k_permute(const uint64_t* __restrict__ n_dev, const uint32_t* __restrict__ sinst,
                          const uint32_t* __restrict__ owner, const float4* __restrict__ r0,
                          const float4* __restrict__ r1, const float4* __restrict__ r2,
                          const float4* __restrict__ r3, float4* __restrict__ s0, float4* __restrict__ s1,
                          float4* __restrict__ s2, float4* __restrict__ s3, uint32_t* __restrict__ sg)
{
    const uint64_t I = *n_dev;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < I; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t g = owner[sinst[i]];
        s0[i] = r0[g]; s1[i] = r1[g]; s2[i] = r2[g]; s3[i] = r3[g];
        sg[i] = g;
    }
}

}  // namespace

gl_status permute_records(View& v, cudaStream_t s)
{
    if (v.I == 0) return GL_OK;
    const size_t I = (size_t)v.I;
    GL_TRY(v.srec0.reserve(16 * I));
    GL_TRY(v.srec1.reserve(16 * I));
    GL_TRY(v.srec2.reserve(16 * I));
    GL_TRY(v.srec3.reserve(16 * I));
    GL_TRY(v.sgid.reserve(4 * I));
    const int blocks = (int)std::min<size_t>(8 * 152, (I + 255) / 256);
    k_permute<<<blocks, 256, 0, s>>>(v.count.as<uint64_t>(), v.sorted_inst, v.iowner.as<uint32_t>(),
                                     v.rec0.as<float4>(), v.rec1.as<float4>(), v.rec2.as<float4>(),
                                     v.rec3.as<float4>(), v.srec0.as<float4>(), v.srec1.as<float4>(),
                                     v.srec2.as<float4>(), v.srec3.as<float4>(), v.sgid.as<uint32_t>());
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

gl_status raster_forward(View& v, float* rgb, float* depth, float* opac, cudaStream_t s)
{
    const size_t P = (size_t)v.P;
    GL_TRY(v.Tfin.reserve(4 * P));
    GL_TRY(v.ncon.reserve(4 * P));
    if (v.ntiles == 0) return GL_OK;
    if (v.Ts != 8 && v.Ts != 16 && v.Ts != 32) { set_error("tile_size must be 8, 16 or 32"); return GL_ERR_INVALID; }
    PhaseScope ps(v.prof, PH_RASTER_FWD, s);
    const int nunits = v.ntiles * (v.Ts * v.Ts / 32);
    const int blocks = (nunits + kWarpsPerBlock - 1) / kWarpsPerBlock;
    k_raster_fwd<<<blocks, 32 * kWarpsPerBlock, 0, s>>>(
        nunits, v.Ts, v.tile_order.as<uint32_t>(), v.ranges.as<uint32_t>(), v.srec0.as<float4>(),
        v.srec1.as<float4>(), v.srec2.as<float4>(), v.srec3.as<float4>(), v.d_desc(), v.V, rgb, depth, opac,
        v.Tfin.as<float>(), v.ncon.as<uint32_t>());
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

gl_status raster_backward(View& v, const float* dL_drgb, const float* dL_ddepth,
                          const float* dL_dopac, cudaStream_t s)
{
    const size_t pairs = (size_t)v.n * v.V;
    GL_TRY(v.g2d.reserve(sizeof(float) * kNG * std::max<size_t>(pairs, 1)));
    PhaseScope ps(v.prof, PH_RASTER_BWD, s);
    GL_CUDA_TRY(cudaMemsetAsync(v.g2d.p, 0, sizeof(float) * kNG * pairs, s));
    if (v.ntiles == 0 || v.I == 0) return GL_OK;
    const bool extra = dL_ddepth != nullptr || dL_dopac != nullptr;
    const int nunits = v.ntiles * (v.Ts * v.Ts / 32);
    const int blocks = (nunits + kWarpsPerBlock - 1) / kWarpsPerBlock;
#define GL_BWD_ARGS                                                                                     \
    nunits, v.Ts, v.tile_order.as<uint32_t>(), v.ranges.as<uint32_t>(), v.srec0.as<float4>(),           \
        v.srec1.as<float4>(), v.srec2.as<float4>(), v.srec3.as<float4>(), v.sgid.as<uint32_t>(), v.d_desc(), \
        v.V, v.Tfin.as<float>(), v.ncon.as<uint32_t>(), dL_drgb, dL_ddepth, dL_dopac, v.g2d.as<float>()
    if (extra) k_raster_bwd<true><<<blocks, 32 * kWarpsPerBlock, 0, s>>>(GL_BWD_ARGS);
    else k_raster_bwd<false><<<blocks, 32 * kWarpsPerBlock, 0, s>>>(GL_BWD_ARGS);
#undef GL_BWD_ARGS
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

}  // namespace gl
