// gl_raster.cu -- front-to-back compositing (Eq. 4-7) and its adjoint.
//
// Work unit: one warp per (screen tile, block of 8 x 4D pixels).  Binning is
// per tile (TS x TS); every pixel block of a tile is rendered by its own
// warp, independently, so a heavy tile is spread over TS*TS/(32 D) warps
// instead of being the critical path of one CTA.  Units are numbered
// heaviest tile first.  Lane l owns the D pixels (x0 + l % 8, y0 + l / 8 + 4 j),
// j < D: the records a warp stages and the warp reduction of the backward are
// shared by D pixels per lane.
//
// Records are permuted into sorted-instance order after binning, so a tile's
// Gaussians are contiguous.  A batch is 32 NB records (NB per lane, the next
// batch prefetched into registers); the warp ballots which records' alpha
// boxes touch its pixel block, compacts the hits in shared memory in depth
// order and evaluates only those.  A Gaussian outside the block's box fails
// the alpha test at every pixel of the block, so skipping it changes no result.
//
// Scheduling: either one unit per warp of a grid that covers all units, or a
// persistent grid (sized to the resident warps) whose warps take the next
// unit from a counter until none is left.
//
// Forward: per pixel, blend until the transmittance would fall below 1e-4;
// keep the final transmittance and the position (in the tile's list) of the
// last blended Gaussian, so the backward recomputes T by division.
// Backward: the same units walked back to front; per hit, each lane sums its
// D pixels' ten partial sums (colour 3, dL/dpower moments 6, depth 1), the
// warp folds the 32 lanes with a transposed butterfly and ten lanes add the
// totals to the Gaussian's accumulator.
#include "gl_internal.h"

namespace gl {

namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kNG = 10;   // screen-space gradient slots per Gaussian

// Inputs shared by the forward and backward kernels (passed by value).
struct RasterArgs {
    int nunits, TS, V;
    const uint32_t* order;       // tiles, heaviest first
    const uint32_t* ranges;      // [first, last + 1) of each tile's list
    const float4 *s0, *s1, *s2, *s3;
    const uint32_t* sgid;        // owning (view, Gaussian) pair of each sorted instance
    const ViewDesc* views;
    int* work;                   // persistent grid: unit counter; nullptr: one unit per warp
};

struct RasterOut {
    float *rgb, *depth, *opac, *Tfin;
    uint32_t* ncon;
};

struct RasterGrad {
    const float* Tfin;
    const uint32_t* ncon;
    const float *dL_drgb, *dL_ddepth, *dL_dopac;
    float* g2d;                  // atomic accumulation per (view, Gaussian)
    // deterministic mode: per (instance, pixel block) sums, indexed by the
    // instance's emission index (sinst of its sorted position)
    float* part;
    const uint32_t* sinst;
    int nblk;                    // pixel blocks per tile
};

struct Unit {
    int wb;                // pixel block within the tile
    int x0, y0;            // absolute pixel origin of the pixel block in its view
    int W, H;              // the view's image size
    long long pix_base;    // the view's first pixel in the concatenated images
    uint32_t rs, re;       // the tile's list
};

template <int D>
__device__ __forceinline__ void unit_of(int u, const RasterArgs& A, Unit& U)
{
    const int TS = A.TS;
    const int wb_per_tile = TS * TS / (32 * D), bpr = TS / 8;
    const int tile = (int)A.order[u / wb_per_tile], wb = u % wb_per_tile;
    U.wb = wb;
    const int v = view_of_tile(A.views, A.V, tile);
    const ViewDesc& d = A.views[v];
    const int lt = tile - d.tile_base;
    U.x0 = (lt % d.TX) * TS + (wb % bpr) * 8;
    U.y0 = (lt / d.TX) * TS + (wb / bpr) * 4 * D;
    U.W = d.cam.W;
    U.H = d.cam.H;
    U.pix_base = d.pix_base;
    U.rs = A.ranges[2 * tile];
    U.re = A.ranges[2 * tile + 1];
}

__device__ __forceinline__ bool box_hit(const float4 box, float bx0, float bx1, float by0, float by1)
{
    return !(box.y < bx0 || box.x > bx1 || box.w < by0 || box.z > by1);
}

// Next unit from the counter (the same value in every lane).
__device__ __forceinline__ int next_unit(int* work, int lane)
{
    int u = 0;
    if (lane == 0) u = atomicAdd(work, 1);
    return __shfl_sync(kFull, u, 0);
}

template <int NB, int D>
__device__ __forceinline__ void fwd_unit(int u, const RasterArgs& A, const RasterOut& O, float4* sr0, float4* sr1,
                                         float4* sr2, uint32_t* spos, int lane)
{
    Unit U;
    unit_of<D>(u, A, U);
    const int x = U.x0 + (lane & 7), y0 = U.y0 + (lane >> 3);
    const float px = (float)x;
    const float bx0 = (float)U.x0, bx1 = (float)(U.x0 + 7), by0 = (float)U.y0, by1 = (float)(U.y0 + 4 * D - 1);
    const unsigned lt = (1u << lane) - 1u;
    float T[D], C0[D], C1[D], C2[D], Dd[D], Oo[D];
    uint32_t last[D];
    bool done[D];
#pragma unroll
    for (int j = 0; j < D; j++) {
        T[j] = 1.0f; C0[j] = C1[j] = C2[j] = Dd[j] = Oo[j] = 0.0f;
        last[j] = 0;
        done[j] = !(x < U.W && y0 + 4 * j < U.H);
    }
    float4 n0[NB], n1[NB], n2[NB], n3[NB];
#pragma unroll
    for (int b = 0; b < NB; b++) {
        const uint32_t i = U.rs + b * 32 + lane;
        if (i < U.re) { n0[b] = A.s0[i]; n1[b] = A.s1[i]; n2[b] = A.s2[i]; n3[b] = A.s3[i]; }
    }
    for (uint32_t base = U.rs; base < U.re; base += 32 * NB) {
        bool lane_done = true;
#pragma unroll
        for (int j = 0; j < D; j++) lane_done = lane_done && done[j];
        if (__all_sync(kFull, lane_done)) break;
        int nh = 0;
#pragma unroll
        for (int b = 0; b < NB; b++) {
            const float4 c0 = n0[b], c1 = n1[b], c2 = n2[b], c3 = n3[b];
            const uint32_t i = base + b * 32 + lane;
            const uint32_t ni = i + 32 * NB;
            if (ni < U.re) { n0[b] = A.s0[ni]; n1[b] = A.s1[ni]; n2[b] = A.s2[ni]; n3[b] = A.s3[ni]; }
            const bool hit = i < U.re && box_hit(c3, bx0, bx1, by0, by1);
            const unsigned mask = __ballot_sync(kFull, hit);
            if (hit) {
                const int k = nh + __popc(mask & lt);
                sr0[k] = c0; sr1[k] = c1; sr2[k] = c2;
                spos[k] = i - U.rs;
            }
            nh += __popc(mask);
        }
        __syncwarp();
        for (int k = 0; k < nh && !lane_done; k++) {
            const float4 a = sr0[k], b = sr1[k];
            bool used = false;
            float wgt[D];
#pragma unroll
            for (int j = 0; j < D; j++) {
                wgt[j] = 0.0f;
                if (done[j]) continue;
                float dx, dy, alpha;
                bool capped;
                if (!pair_eval(a, b, px, (float)(y0 + 4 * j), dx, dy, alpha, capped)) continue;
                const float tT = __fmul_rn(T[j], __fsub_rn(1.0f, alpha));
                if (tT < kTransMin) { done[j] = true; continue; }
                wgt[j] = alpha * T[j];
                T[j] = tT;
                last[j] = spos[k] + 1;
                used = true;
            }
            if (used) {
                const float4 c = sr2[k];
#pragma unroll
                for (int j = 0; j < D; j++) {
                    C0[j] += c.x * wgt[j]; C1[j] += c.y * wgt[j]; C2[j] += c.z * wgt[j];
                    Dd[j] += b.z * wgt[j]; Oo[j] += wgt[j];
                }
            }
            lane_done = true;
#pragma unroll
            for (int j = 0; j < D; j++) lane_done = lane_done && done[j];
        }
        __syncwarp();
    }
#pragma unroll
    for (int j = 0; j < D; j++) {
        const int y = y0 + 4 * j;
        if (!(x < U.W && y < U.H)) continue;
        const size_t p = (size_t)U.pix_base + (size_t)y * U.W + x;
        O.rgb[3 * p] = C0[j]; O.rgb[3 * p + 1] = C1[j]; O.rgb[3 * p + 2] = C2[j];
        if (O.depth) O.depth[p] = Dd[j];
        if (O.opac) O.opac[p] = Oo[j];
        O.Tfin[p] = T[j];
        O.ncon[p] = last[j];
    }
}

template <int NB, int D>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
k_raster_fwd(RasterArgs A, RasterOut O)
{
    __shared__ float4 sr0[kWarpsPerBlock][32 * NB], sr1[kWarpsPerBlock][32 * NB], sr2[kWarpsPerBlock][32 * NB];
    __shared__ uint32_t spos[kWarpsPerBlock][32 * NB];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int u = A.work ? next_unit(A.work, lane) : blockIdx.x * kWarpsPerBlock + w;
    while (u < A.nunits) {
        fwd_unit<NB, D>(u, A, O, sr0[w], sr1[w], sr2[w], spos[w], lane);
        if (!A.work) break;
        u = next_unit(A.work, lane);
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

template <bool EXTRA, int NB, int D, bool DET>
__device__ __forceinline__ void bwd_unit(int u, const RasterArgs& A, const RasterGrad& G, float4* sr0,
                                         float4* sr1, float4* sr2, uint32_t* spos, uint32_t* sg, int lane)
{
    Unit U;
    unit_of<D>(u, A, U);
    const int x = U.x0 + (lane & 7), y0 = U.y0 + (lane >> 3);
    const float px = (float)x;
    const float bx0 = (float)U.x0, bx1 = (float)(U.x0 + 7), by0 = (float)U.y0, by1 = (float)(U.y0 + 4 * D - 1);
    const unsigned lt = (1u << lane) - 1u;
    float T[D], R0[D], R1[D], R2[D], RD[D], RO[D], g0[D], g1[D], g2[D], gD[D], gO[D];
    uint32_t last[D];
    uint32_t wmax = 0;
#pragma unroll
    for (int j = 0; j < D; j++) {
        T[j] = 1.0f; R0[j] = R1[j] = R2[j] = RD[j] = RO[j] = 0.0f;
        g0[j] = g1[j] = g2[j] = gD[j] = gO[j] = 0.0f;
        last[j] = 0;
        const int y = y0 + 4 * j;
        if (x < U.W && y < U.H) {
            const size_t p = (size_t)U.pix_base + (size_t)y * U.W + x;
            T[j] = G.Tfin[p];
            last[j] = G.ncon[p];
            g0[j] = G.dL_drgb[3 * p]; g1[j] = G.dL_drgb[3 * p + 1]; g2[j] = G.dL_drgb[3 * p + 2];
            if (EXTRA) {
                gD[j] = G.dL_ddepth ? G.dL_ddepth[p] : 0.0f;
                gO[j] = G.dL_dopac ? G.dL_dopac[p] : 0.0f;
            }
        }
        wmax = max(wmax, last[j]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wmax = max(wmax, __shfl_xor_sync(kFull, wmax, off));
    const uint32_t end = U.rs + wmax;   // positions at or beyond this reach no pixel of the block
    if (end == U.rs) return;
    // batches from the back: [bstart, bstart + 32 NB) with bstart = end - 32 NB k, clipped at rs
    constexpr int BS = 32 * NB;
    int64_t bstart = (int64_t)end - BS;
    float4 n0[NB], n1[NB], n2[NB], n3[NB];
    uint32_t ng[NB];
#pragma unroll
    for (int b = 0; b < NB; b++) {
        const int64_t i = bstart + b * 32 + lane;
        ng[b] = 0;
        if (i >= (int64_t)U.rs) {
            n0[b] = A.s0[i]; n1[b] = A.s1[i]; n2[b] = A.s2[i]; n3[b] = A.s3[i];
            ng[b] = DET ? G.sinst[i] : A.sgid[i];
        }
    }
    for (; bstart + BS > (int64_t)U.rs; bstart -= BS) {
        int nh = 0;
#pragma unroll
        for (int b = 0; b < NB; b++) {
            const float4 c0 = n0[b], c1 = n1[b], c2 = n2[b], c3 = n3[b];
            const uint32_t cg = ng[b];
            const int64_t i = bstart + b * 32 + lane;
            const int64_t ni = i - BS;
            if (ni >= (int64_t)U.rs) {
                n0[b] = A.s0[ni]; n1[b] = A.s1[ni]; n2[b] = A.s2[ni]; n3[b] = A.s3[ni];
                ng[b] = DET ? G.sinst[ni] : A.sgid[ni];
            }
            const bool hit = i >= (int64_t)U.rs && box_hit(c3, bx0, bx1, by0, by1);
            const unsigned mask = __ballot_sync(kFull, hit);
            if (hit) {
                const int k = nh + __popc(mask & lt);
                sr0[k] = c0; sr1[k] = c1; sr2[k] = c2;
                spos[k] = (uint32_t)(i - U.rs);
                sg[k] = cg;
            }
            nh += __popc(mask);
        }
        __syncwarp();
        for (int k = nh - 1; k >= 0; k--) {
            const float4 a = sr0[k], b = sr1[k], c = sr2[k];
            const uint32_t pos = spos[k];
            float v[16];
#pragma unroll
            for (int q = 0; q < 16; q++) v[q] = 0.0f;
            bool any = false;
#pragma unroll
            for (int j = 0; j < D; j++) {
                float dx, dy, alpha;
                bool capped;
                if (pos < last[j] && pair_eval(a, b, px, (float)(y0 + 4 * j), dx, dy, alpha, capped)) {
                    const float om = 1.0f - alpha;
                    T[j] = __fdividef(T[j], om);
                    const float wgt = alpha * T[j];
                    float ga = g0[j] * (c.x - R0[j]) + g1[j] * (c.y - R1[j]) + g2[j] * (c.z - R2[j]);
                    if (EXTRA) ga += gD[j] * (b.z - RD[j]) + gO[j] * (1.0f - RO[j]);
                    ga *= T[j];
                    R0[j] = alpha * c.x + om * R0[j];
                    R1[j] = alpha * c.y + om * R1[j];
                    R2[j] = alpha * c.z + om * R2[j];
                    if (EXTRA) {
                        RD[j] = alpha * b.z + om * RD[j];
                        RO[j] = alpha + om * RO[j];
                    }
                    const float gp = capped ? 0.0f : ga * alpha;
                    v[0] += wgt * g0[j]; v[1] += wgt * g1[j]; v[2] += wgt * g2[j];
                    v[3] += gp;
                    v[4] += gp * dx; v[5] += gp * dy;
                    v[6] += gp * dx * dx; v[7] += gp * dx * dy; v[8] += gp * dy * dy;
                    if (EXTRA) v[9] += wgt * gD[j];
                    any = true;
                }
            }
            if (__any_sync(kFull, any)) {
                const float r = warp_transpose_reduce16(v);
                const int q = lane >> 1;
                if ((lane & 1) == 0 && q < (EXTRA ? kNG : kNG - 1)) {
                    if (DET) G.part[((size_t)sg[k] * G.nblk + U.wb) * kNG + q] = r;
                    else atomicAdd(G.g2d + (size_t)sg[k] * kNG + q, r);
                }
            }
        }
        __syncwarp();
    }
}

template <bool EXTRA, int NB, int D, bool DET>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
k_raster_bwd(RasterArgs A, RasterGrad G)
{
    __shared__ float4 sr0[kWarpsPerBlock][32 * NB], sr1[kWarpsPerBlock][32 * NB], sr2[kWarpsPerBlock][32 * NB];
    __shared__ uint32_t spos[kWarpsPerBlock][32 * NB], sg[kWarpsPerBlock][32 * NB];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int u = A.work ? next_unit(A.work, lane) : blockIdx.x * kWarpsPerBlock + w;
    while (u < A.nunits) {
        bwd_unit<EXTRA, NB, D, DET>(u, A, G, sr0[w], sr1[w], sr2[w], spos[w], sg[w], lane);
        if (!A.work) break;
        u = next_unit(A.work, lane);
    }
}

// Deterministic gradient sums: for each (view, Gaussian) pair, its instances
// (emission indices dup_off .. dup_off + touched) and each instance's pixel
// blocks in ascending order.
__global__ void k_part_reduce(const float* __restrict__ part, const uint32_t* __restrict__ touched,
                              const uint32_t* __restrict__ dup_off, int nblk, int64_t pairs,
                              const uint64_t* __restrict__ ctl, uint64_t cap, float* __restrict__ g2d)
{
    const bool overflow = ctl[1] != 0;   // the step's instances did not fit: nothing was written
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < pairs;
         t += (int64_t)gridDim.x * blockDim.x) {
        float acc[kNG];
#pragma unroll
        for (int q = 0; q < kNG; q++) acc[q] = 0.0f;
        const uint32_t cnt = touched[t];
        if (cnt && !overflow && (uint64_t)dup_off[t] + cnt <= cap) {
            const float* p = part + (size_t)dup_off[t] * nblk * kNG;
            for (uint32_t e = 0; e < cnt * (uint32_t)nblk; e++, p += kNG) {
#pragma unroll
                for (int q = 0; q < kNG; q++) acc[q] += p[q];
            }
        }
#pragma unroll
        for (int q = 0; q < kNG; q++) g2d[(size_t)t * kNG + q] = acc[q];
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

template <typename K>
int grid_for(K kernel, int variant, int nunits, bool persistent)
{
    const int need = (nunits + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (!persistent) return need;
    // resident CTAs of this variant, looked up once per process
    static int cache[64] = {};
    if (!cache[variant]) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 32 * kWarpsPerBlock, 0);
        cache[variant] = std::max(1, sms * std::max(1, per));
    }
    return std::max(1, std::min(need, cache[variant]));
}

RasterArgs make_args(View& v, int* work)
{
    RasterArgs A;
    A.nunits = v.ntiles * (v.Ts * v.Ts / (32 * v.pd));
    A.TS = v.Ts;
    A.V = v.V;
    A.order = v.tile_order.as<uint32_t>();
    A.ranges = v.ranges.as<uint32_t>();
    A.s0 = v.srec0.as<float4>();
    A.s1 = v.srec1.as<float4>();
    A.s2 = v.srec2.as<float4>();
    A.s3 = v.srec3.as<float4>();
    A.sgid = v.sgid.as<uint32_t>();
    A.views = v.d_desc();
    A.work = work;
    return A;
}

gl_status check_exec(const View& v)
{
    if (v.Ts != 8 && v.Ts != 16 && v.Ts != 32) { set_error("tile_size must be 8, 16 or 32"); return GL_ERR_INVALID; }
    if (v.nb != 1 && v.nb != 2) { set_error("batch depth must be 32 or 64"); return GL_ERR_INVALID; }
    if ((v.pd != 1 && v.pd != 2 && v.pd != 4) || 4 * v.pd > v.Ts) {
        set_error("pixels per lane must be 1, 2 or 4, with 4 x pixels per lane <= tile size");
        return GL_ERR_INVALID;
    }
    return GL_OK;
}

template <int NB, int D>
void fwd_launch(const RasterArgs& A, const RasterOut& O, bool persistent, cudaStream_t s)
{
    const int grid = grid_for(k_raster_fwd<NB, D>, (NB - 1) * 4 + D, A.nunits, persistent);
    k_raster_fwd<NB, D><<<grid, 32 * kWarpsPerBlock, 0, s>>>(A, O);
}

template <bool EXTRA, int NB, int D, bool DET>
void bwd_launch(const RasterArgs& A, const RasterGrad& G, bool persistent, cudaStream_t s)
{
    const int variant = 32 + (DET ? 16 : 0) + (EXTRA ? 8 : 0) + (NB - 1) * 4 + D;   // < 64
    const int grid = grid_for(k_raster_bwd<EXTRA, NB, D, DET>, variant, A.nunits, persistent);
    k_raster_bwd<EXTRA, NB, D, DET><<<grid, 32 * kWarpsPerBlock, 0, s>>>(A, G);
}

template <bool EXTRA>
void bwd_dispatch(int nb, int pd, bool det, const RasterArgs& A, const RasterGrad& G, bool persistent,
                  cudaStream_t s)
{
    if (det) {   // batch depth 32 only
        if (pd == 1) bwd_launch<EXTRA, 1, 1, true>(A, G, persistent, s);
        else if (pd == 2) bwd_launch<EXTRA, 1, 2, true>(A, G, persistent, s);
        else bwd_launch<EXTRA, 1, 4, true>(A, G, persistent, s);
    } else if (nb == 1) {
        if (pd == 1) bwd_launch<EXTRA, 1, 1, false>(A, G, persistent, s);
        else if (pd == 2) bwd_launch<EXTRA, 1, 2, false>(A, G, persistent, s);
        else bwd_launch<EXTRA, 1, 4, false>(A, G, persistent, s);
    } else {
        if (pd == 1) bwd_launch<EXTRA, 2, 1, false>(A, G, persistent, s);
        else if (pd == 2) bwd_launch<EXTRA, 2, 2, false>(A, G, persistent, s);
        else bwd_launch<EXTRA, 2, 4, false>(A, G, persistent, s);
    }
}

}  // namespace

gl_status permute_records(View& v, int64_t nmax, cudaStream_t s)
{
    if (nmax <= 0) return GL_OK;
    const size_t I = (size_t)nmax;
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
    GL_TRY(check_exec(v));
    GL_TRY(v.work.reserve(16));
    PhaseScope ps(v.prof, PH_RASTER_FWD, s);
    int* work = nullptr;
    if (v.persistent) {
        work = v.work.as<int>();
        GL_CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(int), s));
    }
    const RasterArgs A = make_args(v, work);
    RasterOut O{rgb, depth, opac, v.Tfin.as<float>(), v.ncon.as<uint32_t>()};
    if (v.nb == 1) {
        if (v.pd == 1) fwd_launch<1, 1>(A, O, v.persistent, s);
        else if (v.pd == 2) fwd_launch<1, 2>(A, O, v.persistent, s);
        else fwd_launch<1, 4>(A, O, v.persistent, s);
    } else {
        if (v.pd == 1) fwd_launch<2, 1>(A, O, v.persistent, s);
        else if (v.pd == 2) fwd_launch<2, 2>(A, O, v.persistent, s);
        else fwd_launch<2, 4>(A, O, v.persistent, s);
    }
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

gl_status raster_backward(View& v, const float* dL_drgb, const float* dL_ddepth,
                          const float* dL_dopac, cudaStream_t s)
{
    const size_t pairs = (size_t)v.n * v.V;
    GL_TRY(v.g2d.reserve(sizeof(float) * kNG * std::max<size_t>(pairs, 1)));
    GL_TRY(check_exec(v));
    GL_TRY(v.work.reserve(16));
    PhaseScope ps(v.prof, PH_RASTER_BWD, s);
    const bool det = v.det && v.ntiles > 0 && v.I != 0;
    const int nblk = v.Ts * v.Ts / (32 * v.pd);
    if (!det) GL_CUDA_TRY(cudaMemsetAsync(v.g2d.p, 0, sizeof(float) * kNG * pairs, s));
    if (v.ntiles == 0 || v.I == 0) return GL_OK;
    int* work = nullptr;
    if (v.persistent) {
        work = v.work.as<int>() + 1;
        GL_CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(int), s));
    }
    const RasterArgs A = make_args(v, work);
    RasterGrad G{v.Tfin.as<float>(), v.ncon.as<uint32_t>(), dL_drgb, dL_ddepth, dL_dopac, v.g2d.as<float>(),
                 nullptr, v.sorted_inst, nblk};
    const size_t cap = v.itile.bytes / 4;
    if (det) {
        // every instance's block sums, zero where a block has no hit; the
        // instance count is bounded by the capacity when it is known on the
        // device only
        const size_t inst = v.I > 0 ? (size_t)v.I : cap;
        GL_TRY(v.gpart.reserve(sizeof(float) * kNG * (size_t)nblk * std::max<size_t>(cap, 1)));
        GL_CUDA_TRY(cudaMemsetAsync(v.gpart.p, 0, sizeof(float) * kNG * (size_t)nblk * inst, s));
        G.part = v.gpart.as<float>();
    }
    if (dL_ddepth != nullptr || dL_dopac != nullptr) bwd_dispatch<true>(v.nb, v.pd, det, A, G, v.persistent, s);
    else bwd_dispatch<false>(v.nb, v.pd, det, A, G, v.persistent, s);
    count_launches(1);
    if (det) {
        const int blocks = (int)std::min<size_t>(8 * 152, (pairs + 255) / 256);
        k_part_reduce<<<std::max(blocks, 1), 256, 0, s>>>(v.gpart.as<float>(), v.touched.as<uint32_t>(),
                                                          v.dup_off.as<uint32_t>(), nblk, (int64_t)pairs,
                                                          v.count.as<uint64_t>(), (uint64_t)cap, v.g2d.as<float>());
        count_launches(1);
    }
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

}  // namespace gl
