// gl_raster.cu -- front-to-back compositing (Eq. 4-7) and its adjoint.
//
// Work unit: one warp per (work item, block of 8 x 4D pixels).  A work item
// is a screen tile (TS x TS) or, for a tile whose list holds at least 2 seg
// records, one segment of seg consecutive records of that list.  Every
// pixel block of a tile is rendered by its own warp, and a long list is
// split along depth, so neither a heavy tile nor a deep one (the road's
// vanishing point gathers tens of thousands of far Gaussians in a few
// tiles) is the critical path of one warp.  Items are numbered heaviest
// first.  Lane l owns the D pixels (x0 + l % 8, y0 + l / 8 + 4 j), j < D:
// the records a warp stages and the warp reduction of the backward are
// shared by D pixels per lane.
//
// Records are permuted into sorted-instance order after binning, so a
// tile's Gaussians are contiguous: a batch is 32 NB records (NB per lane, the
// next batch prefetched into registers); the warp ballots which records'
// alpha boxes touch its pixel block, compacts the hits in shared memory in
// depth order and evaluates only those.  A Gaussian outside the block's box
// fails the alpha test at every pixel of the block, so skipping it changes
// no result.
//
// Forward of a whole tile: per pixel, blend until the transmittance would
// fall below 1e-4; keep the final transmittance and the position (in the
// tile's list) of the last blended Gaussian, so the backward recomputes T by
// division.
//
// Forward of a split tile, in four launches.  (1) Each segment item blends
// its records per pixel from T = 1 without the stop rule and stores the
// segment's transmittance product T_s, colour, depth and opacity sums and
// last blended position.  (2) A prefix pass walks each pixel's segments in
// order with the incoming transmittance T_in (the product of the earlier
// T_s): the stop rule fires inside segment s exactly when T_in * T_s falls
// below 1e-4 (the running value inside s is T_in times the segment's own
// running product, and that product only decreases).  (3) Each segment
// item replays its records from T_in for the pixels that stop in it (one
// replay per warp, all segments in parallel) to find the stop and the
// truncated sums.  (4) A finish pass writes the pixel's outputs and, per
// segment, the backward's starting state: the transmittance after the
// segment and the normalised colour blended behind it (R = C_next + T_next
// * R_next over the later segments).
// The transmittance is the product of the per-segment products, so it can
// differ from a single running product by float rounding.
//
// Backward: every item walked back to front from its starting state (the
// final transmittance and R = 0 for a whole tile); per hit, each lane sums
// its D pixels' ten partial sums (colour 3, dL/dpower moments 6, depth 1),
// the warp folds the 32 lanes with a transposed butterfly and ten lanes add
// the totals to the Gaussian's accumulator (or, deterministic, store them
// per instance and pixel block).
//
// Scheduling: either one unit per warp of a grid that covers the bound on
// units, or a persistent grid (sized to the resident warps) whose warps take
// the next unit from a counter; the number of units is read on the device.
#include "gl_internal.h"

#include <map>
#include <mutex>

namespace gl {

namespace {

constexpr int kWarpsPerBlock = 8;
// Warps per CTA of the kernels that stage 32 NB records per warp: batches of
// 128 and 256 records use 4 and 2 warps, so that every variant's staged hits
// fit in 48 KB of shared memory with the same resident warps per SM.
template <int NB>
constexpr int wpb() { return NB <= 2 ? kWarpsPerBlock : 16 / NB; }
// Prefetch slots (32 records each) of a batch of 32 NB records: the whole
// next batch up to 64 records, one sub-batch ahead beyond.
template <int NB>
constexpr int pf_slots() { return NB <= 2 ? NB : 1; }
// resident CTAs per SM the kernels are compiled for: the forward passes fit
// 64 registers (4 CTAs); the backward is faster with 76 registers (3 CTAs)
// than squeezed into 64
constexpr int kMinBlocks = 4;
constexpr int kMinBlocksBwd = 3;
constexpr int kNG = 10;   // screen-space gradient slots per Gaussian
constexpr int kSegFields = 16;  // per (segment item, pixel): see below
constexpr int kSegBatch = 4;    // segments whose state one load round trip brings (prefix, finish)

// segstate fields of a segment item.  After the segment pass: 0 T_s, 1-3
// colour, 4 depth, 5 opacity, 6 last position (as bits); 7 the incoming
// transmittance (prefix pass); fields 0-6 replaced by the truncated sums in
// the segment where the pixel stops (replay pass).  After the finish pass:
// 0 transmittance after the segment, 1-3 R (colour behind it, normalised),
// 4 R depth, 5 R opacity.  Fields 8-15 of a split tile's first item hold the
// tile-level state of the pixel: 8 stop segment (bits; segments = none),
// 9 transmittance entering it (or the final one), 10-12 colour, 13 depth,
// 14 opacity summed over the segments before it, 15 last position there.
__device__ __forceinline__ size_t seg_at(int w, int k, int p, int TS)
{
    return ((size_t)w * kSegFields + k) * (size_t)(TS * TS) + p;
}

// Inputs shared by the kernels (passed by value).
struct RasterArgs {
    int TS, V, nblk, seg;
    const uint2* items;          // (tile, segment), heaviest first
    const uint64_t* ctl;         // ctl[6] work items, ctl[7] items of split tiles
    const uint32_t* ranges;      // [first, last + 1) of each tile's list
    const float4 *s0, *s1, *s2, *s3;
    const uint32_t* sgid;        // owning (view, Gaussian) pair of each sorted instance
    const ViewDesc* views;
    float* segstate;
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
};

struct Unit {
    int w, wb;             // work item, pixel block within the tile
    int j, nseg;           // segment of the item and segments of its tile
    int lx0, ly0;          // pixel block origin within the tile
    int x0, y0;            // absolute pixel origin of the pixel block in its view
    int W, H;              // the view's image size
    long long pix_base;    // the view's first pixel in the concatenated images
    uint32_t trs, tre;     // the tile's whole list
    uint32_t rs, re;       // the item's part of it
};

template <int D>
__device__ __forceinline__ void unit_of(int u, const RasterArgs& A, Unit& U)
{
    // pixel blocks per tile, blocks per tile row and the segment length are
    // powers of two: shifts and masks instead of integer divisions
    const int TS = A.TS, bsh = __ffs(TS >> 3) - 1, nsh = __ffs(A.nblk) - 1;
    U.w = u >> nsh;
    U.wb = u & (A.nblk - 1);
    const uint2 it = A.items[U.w];
    const int tile = (int)it.x;
    U.j = (int)it.y;
    const int v = view_of_tile(A.views, A.V, tile);
    const ViewDesc& d = A.views[v];
    const int lt = tile - d.tile_base;
    U.lx0 = (U.wb & ((1 << bsh) - 1)) * 8;
    U.ly0 = (U.wb >> bsh) * 4 * D;
    U.x0 = (lt % d.TX) * TS + U.lx0;
    U.y0 = (lt / d.TX) * TS + U.ly0;
    U.W = d.cam.W;
    U.H = d.cam.H;
    U.pix_base = d.pix_base;
    U.trs = A.ranges[2 * tile];
    U.tre = A.ranges[2 * tile + 1];
    const uint32_t L = U.tre - U.trs;
    U.nseg = (A.seg > 0 && L >= 2u * (uint32_t)A.seg) ? (int)((L + A.seg - 1) >> (__ffs(A.seg) - 1)) : 1;
    if (U.nseg > 1) {
        U.rs = U.trs + (uint32_t)U.j * (uint32_t)A.seg;
        U.re = min(U.tre, U.rs + (uint32_t)A.seg);
    } else {
        U.rs = U.trs;
        U.re = U.tre;
    }
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

// Units of this launch: work items (or the split tiles' items) x pixel blocks.
__device__ __forceinline__ int units_of(const RasterArgs& A, bool split_only)
{
    return (int)(A.ctl[split_only ? 7 : 6]) * A.nblk;
}

// Front-to-back blend of the records [a, b) of a tile list for the warp's
// pixel block.  Per pixel: T (running transmittance), colour, depth and
// opacity sums (XD; without it they stay 0) and the last blended position
// (relative to trs).  With `stop`, a pixel stops (without blending) at the
// first record whose T * (1 - alpha), scaled by its Tin, falls below 1e-4;
// without it every accepted record is blended and a pixel stops only when T
// reaches 0.  Pixels with done set take no part.
template <int NB, int D, bool XD>
__device__ __forceinline__ void blend_range(const RasterArgs& A, uint32_t a, uint32_t b, uint32_t trs, float px,
                                            const float (&py)[D], float bx0, float bx1, float by0, float by1,
                                            bool stop, const float (&Tin)[D], bool (&done)[D], float (&T)[D],
                                            float (&C0)[D], float (&C1)[D], float (&C2)[D], float (&Dd)[D],
                                            float (&Oo)[D], uint32_t (&last)[D], float4* sr0, float4* sr1,
                                            float4* sr2, uint32_t* spos, int lane)
{
    const unsigned lt = (1u << lane) - 1u;
    constexpr int PF = pf_slots<NB>();
    float4 n0[PF], n1[PF], n2[PF], n3[PF];
#pragma unroll
    for (int q = 0; q < PF; q++) {
        const uint32_t i = a + q * 32 + lane;
        if (i < b) { n0[q] = A.s0[i]; n1[q] = A.s1[i]; n2[q] = A.s2[i]; n3[q] = A.s3[i]; }
    }
    for (uint32_t base = a; base < b; base += 32 * NB) {
        bool lane_done = true;
#pragma unroll
        for (int j = 0; j < D; j++) lane_done = lane_done && done[j];
        if (__all_sync(kFull, lane_done)) break;
        int nh = 0;
#pragma unroll
        for (int q = 0; q < NB; q++) {
            const int sl = PF == NB ? q : 0;
            const float4 c0 = n0[sl], c1 = n1[sl], c2 = n2[sl], c3 = n3[sl];
            const uint32_t i = base + q * 32 + lane;
            const uint32_t ni = i + 32 * PF;
            if (ni < b) { n0[sl] = A.s0[ni]; n1[sl] = A.s1[ni]; n2[sl] = A.s2[ni]; n3[sl] = A.s3[ni]; }
            const bool hit = i < b && box_hit(c3, bx0, bx1, by0, by1);
            const unsigned mask = __ballot_sync(kFull, hit);
            if (hit) {
                const int k = nh + __popc(mask & lt);
                sr0[k] = c0; sr1[k] = c1; sr2[k] = c2;
                spos[k] = i - trs;
            }
            nh += __popc(mask);
        }
        __syncwarp();
        for (int k = 0; k < nh && !lane_done; k++) {
            // Branch-free: a pixel that is done, or that the hit misses or
            // stops at, blends with weight 0 (its sums exactly unchanged);
            // T and the last position move by selects.
            const float4 g0 = sr0[k], g1 = sr1[k], c = sr2[k];
            const uint32_t pos1 = spos[k] + 1;
#pragma unroll
            for (int j = 0; j < D; j++) {
                float dx, dy, alpha;
                bool capped;
                const bool live = pair_eval_nb(g0, g1, px, py[j], dx, dy, alpha, capped) && !done[j];
                const float tT = __fmul_rn(T[j], __fsub_rn(1.0f, alpha));
                const bool halt = stop && live && __fmul_rn(Tin[j], tT) < kTransMin;
                const bool blend = live && !halt;
                const float wgt = blend ? alpha * T[j] : 0.0f;
                T[j] = blend ? tT : T[j];
                last[j] = blend ? pos1 : last[j];
                done[j] = done[j] || halt || (!stop && blend && tT == 0.0f);
                C0[j] += c.x * wgt; C1[j] += c.y * wgt; C2[j] += c.z * wgt;
                if (XD) {
                    Dd[j] += g1.z * wgt;
                    Oo[j] += wgt;
                }
            }
            lane_done = true;
#pragma unroll
            for (int j = 0; j < D; j++) lane_done = lane_done && done[j];
        }
        __syncwarp();
    }
}

// Per-lane pixel geometry of a unit.
template <int D>
struct LanePix {
    int x;
    float px, py[D];   // relative to the tile's origin, as the records' means
    bool inside[D];
    int p[D];          // pixel index within the tile
    float bx0, bx1, by0, by1;
    __device__ __forceinline__ LanePix(const Unit& U, int TS, int lane)
    {
        x = U.x0 + (lane & 7);
        px = (float)(U.lx0 + (lane & 7));
#pragma unroll
        for (int j = 0; j < D; j++) {
            const int y = U.y0 + (lane >> 3) + 4 * j;
            py[j] = (float)(U.ly0 + (lane >> 3) + 4 * j);
            inside[j] = x < U.W && y < U.H;
            p[j] = (U.ly0 + (lane >> 3) + 4 * j) * TS + U.lx0 + (lane & 7);
        }
        bx0 = (float)U.x0;
        bx1 = (float)(U.x0 + 7);
        by0 = (float)U.y0;
        by1 = (float)(U.y0 + 4 * D - 1);
    }
    __device__ __forceinline__ size_t pix(const Unit& U, int j) const
    {
        return (size_t)U.pix_base + (size_t)(U.y0 + (threadIdx.x & 31) / 8 + 4 * j) * U.W + x;
    }
};

template <int NB, int D, bool XD>
__device__ __forceinline__ void fwd_item(int u, const RasterArgs& A, const RasterOut& O, float4* sr0, float4* sr1,
                                         float4* sr2, uint32_t* spos, int lane)
{
    Unit U;
    unit_of<D>(u, A, U);
    const LanePix<D> L(U, A.TS, lane);
    float T[D], C0[D], C1[D], C2[D], Dd[D], Oo[D], one[D];
    uint32_t last[D];
    bool done[D];
#pragma unroll
    for (int j = 0; j < D; j++) {
        T[j] = 1.0f; C0[j] = C1[j] = C2[j] = Dd[j] = Oo[j] = 0.0f;
        one[j] = 1.0f;
        last[j] = 0;
        done[j] = !L.inside[j];
    }
    const bool whole = U.nseg == 1;
    blend_range<NB, D, XD>(A, U.rs, U.re, U.trs, L.px, L.py, L.bx0, L.bx1, L.by0, L.by1, whole, one, done, T, C0, C1,
                           C2, Dd, Oo, last, sr0, sr1, sr2, spos, lane);
#pragma unroll
    for (int j = 0; j < D; j++) {
        if (!L.inside[j]) continue;
        if (whole) {
            const size_t p = L.pix(U, j);
            O.rgb[3 * p] = C0[j]; O.rgb[3 * p + 1] = C1[j]; O.rgb[3 * p + 2] = C2[j];
            if (O.depth) O.depth[p] = Dd[j];
            if (O.opac) O.opac[p] = Oo[j];
            O.Tfin[p] = T[j];
            O.ncon[p] = last[j];
        } else {
            float* S = A.segstate;
            const int q = L.p[j];
            S[seg_at(U.w, 0, q, A.TS)] = T[j];
            S[seg_at(U.w, 1, q, A.TS)] = C0[j];
            S[seg_at(U.w, 2, q, A.TS)] = C1[j];
            S[seg_at(U.w, 3, q, A.TS)] = C2[j];
            S[seg_at(U.w, 4, q, A.TS)] = Dd[j];
            S[seg_at(U.w, 5, q, A.TS)] = Oo[j];
            S[seg_at(U.w, 6, q, A.TS)] = __uint_as_float(last[j]);
        }
    }
}

template <int NB, int D, bool XD>
__global__ void __launch_bounds__(32 * wpb<NB>(), kMinBlocks * kWarpsPerBlock / wpb<NB>())
k_raster_fwd(RasterArgs A, RasterOut O)
{
    constexpr int WPB = wpb<NB>();
    __shared__ float4 sr0[WPB][32 * NB], sr1[WPB][32 * NB], sr2[WPB][32 * NB];
    __shared__ uint32_t spos[WPB][32 * NB];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nunits = units_of(A, false);
    int u = A.work ? next_unit(A.work, lane) : blockIdx.x * WPB + w;
    while (u < nunits) {
        fwd_item<NB, D, XD>(u, A, O, sr0[w], sr1[w], sr2[w], spos[w], lane);
        if (!A.work) break;
        u = next_unit(A.work, lane);
    }
}

// Split tiles, pass 2 of 4 (after the segment pass): per pixel of a split
// tile, the prefix of its segments' transmittance, the segment where the
// stop rule fires (T_in * T_s < 1e-4) and the sums before it.
template <int D>
__device__ __forceinline__ void prefix_item(int u, const RasterArgs& A, int lane)
{
    Unit U;
    unit_of<D>(u, A, U);
    if (U.j != 0 || U.nseg < 2) return;
    const LanePix<D> L(U, A.TS, lane);
    const int w0 = U.w, ns = U.nseg, TS = A.TS;
    float* S = A.segstate;
#pragma unroll
    for (int j = 0; j < D; j++) {
        if (!L.inside[j]) continue;
        const int q = L.p[j];
        float Tb = 1.0f, c0 = 0.f, c1 = 0.f, c2 = 0.f, dd = 0.f, oo = 0.f;
        uint32_t last = 0;
        int stop = ns;
        // the seven fields of kSegBatch segments are loaded before any of
        // them is used, so that the serial walk waits for memory once per
        // kSegBatch segments
        for (int s0 = 0; s0 < ns && stop == ns; s0 += kSegBatch) {
            float f[kSegBatch][7];
#pragma unroll
            for (int b = 0; b < kSegBatch; b++)
                if (s0 + b < ns) {
#pragma unroll
                    for (int k = 0; k < 7; k++) f[b][k] = S[seg_at(w0 + s0 + b, k, q, TS)];
                }
#pragma unroll
            for (int b = 0; b < kSegBatch; b++) {
                const int s = s0 + b;
                if (s >= ns || stop != ns) break;
                const float Ts = f[b][0];
                S[seg_at(w0 + s, 7, q, TS)] = Tb;
                if (__fmul_rn(Tb, Ts) < kTransMin) { stop = s; break; }
                c0 += Tb * f[b][1];
                c1 += Tb * f[b][2];
                c2 += Tb * f[b][3];
                dd += Tb * f[b][4];
                oo += Tb * f[b][5];
                const uint32_t ls = __float_as_uint(f[b][6]);
                if (ls) last = ls;
                Tb = __fmul_rn(Tb, Ts);
            }
        }
        S[seg_at(w0, 8, q, TS)] = __uint_as_float((uint32_t)stop);
        S[seg_at(w0, 9, q, TS)] = Tb;
        S[seg_at(w0, 10, q, TS)] = c0;
        S[seg_at(w0, 11, q, TS)] = c1;
        S[seg_at(w0, 12, q, TS)] = c2;
        S[seg_at(w0, 13, q, TS)] = dd;
        S[seg_at(w0, 14, q, TS)] = oo;
        S[seg_at(w0, 15, q, TS)] = __uint_as_float(last);
    }
}

// Split tiles, pass 3 of 4: each segment item replays its records from the
// incoming transmittance for the pixels whose stop segment it is, and stores
// their truncated sums in place of the segment pass's.
template <int NB, int D, bool XD>
__device__ __forceinline__ void replay_item(int u, const RasterArgs& A, float4* sr0, float4* sr1, float4* sr2,
                                            uint32_t* spos, int lane)
{
    Unit U;
    unit_of<D>(u, A, U);
    if (U.nseg < 2) return;
    const LanePix<D> L(U, A.TS, lane);
    const int w0 = U.w - U.j, TS = A.TS;
    float* S = A.segstate;
    float Tin[D], T[D], c0[D], c1[D], c2[D], dd[D], oo[D];
    uint32_t last[D];
    bool dn[D];
    bool any = false;
#pragma unroll
    for (int j = 0; j < D; j++) {
        T[j] = 1.0f; c0[j] = c1[j] = c2[j] = dd[j] = oo[j] = 0.0f;
        last[j] = 0;
        Tin[j] = 1.0f;
        dn[j] = true;
        if (!L.inside[j]) continue;
        const int q = L.p[j];
        if ((int)__float_as_uint(S[seg_at(w0, 8, q, TS)]) != U.j) continue;
        Tin[j] = S[seg_at(w0, 9, q, TS)];
        dn[j] = false;
        any = true;
    }
    if (!__any_sync(kFull, any)) return;
    blend_range<NB, D, XD>(A, U.rs, U.re, U.trs, L.px, L.py, L.bx0, L.bx1, L.by0, L.by1, true, Tin, dn, T, c0, c1,
                           c2, dd, oo, last, sr0, sr1, sr2, spos, lane);
#pragma unroll
    for (int j = 0; j < D; j++) {
        if (!L.inside[j]) continue;
        const int q = L.p[j];
        if ((int)__float_as_uint(S[seg_at(w0, 8, q, TS)]) != U.j) continue;
        S[seg_at(U.w, 0, q, TS)] = T[j];
        S[seg_at(U.w, 1, q, TS)] = c0[j];
        S[seg_at(U.w, 2, q, TS)] = c1[j];
        S[seg_at(U.w, 3, q, TS)] = c2[j];
        S[seg_at(U.w, 4, q, TS)] = dd[j];
        S[seg_at(U.w, 5, q, TS)] = oo[j];
        S[seg_at(U.w, 6, q, TS)] = __uint_as_float(last[j]);
    }
}

// Split tiles, pass 4 of 4: per pixel, the outputs (sums before the stop
// segment plus its truncated sums) and, back to front over the segments up
// to the stop, the backward's starting state of each.
template <int D>
__device__ __forceinline__ void finish_item(int u, const RasterArgs& A, const RasterOut& O, int lane)
{
    Unit U;
    unit_of<D>(u, A, U);
    if (U.j != 0 || U.nseg < 2) return;
    const LanePix<D> L(U, A.TS, lane);
    const int w0 = U.w, ns = U.nseg, TS = A.TS;
    float* S = A.segstate;
#pragma unroll
    for (int j = 0; j < D; j++) {
        if (!L.inside[j]) continue;
        const int q = L.p[j];
        const int stop = (int)__float_as_uint(S[seg_at(w0, 8, q, TS)]);
        float Tb = S[seg_at(w0, 9, q, TS)];
        float c0 = S[seg_at(w0, 10, q, TS)], c1 = S[seg_at(w0, 11, q, TS)], c2 = S[seg_at(w0, 12, q, TS)];
        float dd = S[seg_at(w0, 13, q, TS)], oo = S[seg_at(w0, 14, q, TS)];
        uint32_t last = __float_as_uint(S[seg_at(w0, 15, q, TS)]);
        if (stop < ns) {
            const int ws = w0 + stop;
            c0 += Tb * S[seg_at(ws, 1, q, TS)];
            c1 += Tb * S[seg_at(ws, 2, q, TS)];
            c2 += Tb * S[seg_at(ws, 3, q, TS)];
            dd += Tb * S[seg_at(ws, 4, q, TS)];
            oo += Tb * S[seg_at(ws, 5, q, TS)];
            const uint32_t ls = __float_as_uint(S[seg_at(ws, 6, q, TS)]);
            if (ls) last = ls;
            Tb = __fmul_rn(Tb, S[seg_at(ws, 0, q, TS)]);
        }
        const size_t p = L.pix(U, j);
        O.rgb[3 * p] = c0; O.rgb[3 * p + 1] = c1; O.rgb[3 * p + 2] = c2;
        if (O.depth) O.depth[p] = dd;
        if (O.opac) O.opac[p] = oo;
        O.Tfin[p] = Tb;
        O.ncon[p] = last;
        const int jl = stop < ns ? stop : ns - 1;
        for (int s = ns - 1; s > jl; s--)
            for (int k = 0; k < 6; k++) S[seg_at(w0 + s, k, q, TS)] = 0.0f;
        // back to front from the stop segment; the fields (0-5 and the
        // incoming transmittance, 7) of kSegBatch segments are loaded before
        // any of them is used
        float R0 = 0.f, R1 = 0.f, R2 = 0.f, RD = 0.f, RO = 0.f;
        for (int s0 = jl; s0 >= 0; s0 -= kSegBatch) {
            float f[kSegBatch][7];
#pragma unroll
            for (int b = 0; b < kSegBatch; b++)
                if (s0 - b >= 0) {
#pragma unroll
                    for (int k = 0; k < 6; k++) f[b][k] = S[seg_at(w0 + s0 - b, k, q, TS)];
                    f[b][6] = S[seg_at(w0 + s0 - b, 7, q, TS)];
                }
#pragma unroll
            for (int b = 0; b < kSegBatch; b++) {
                const int s = s0 - b;
                if (s < 0) break;
                const int ws = w0 + s;
                const float Ts = f[b][0], cs0 = f[b][1], cs1 = f[b][2], cs2 = f[b][3], ds = f[b][4], os = f[b][5];
                const float tin = f[b][6];
                S[seg_at(ws, 0, q, TS)] = __fmul_rn(tin, Ts);
                S[seg_at(ws, 1, q, TS)] = R0;
                S[seg_at(ws, 2, q, TS)] = R1;
                S[seg_at(ws, 3, q, TS)] = R2;
                S[seg_at(ws, 4, q, TS)] = RD;
                S[seg_at(ws, 5, q, TS)] = RO;
                R0 = cs0 + Ts * R0; R1 = cs1 + Ts * R1; R2 = cs2 + Ts * R2;
                RD = ds + Ts * RD; RO = os + Ts * RO;
            }
        }
    }
}

template <int D>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, kMinBlocks) k_seg_prefix(RasterArgs A)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nunits = units_of(A, true);
    int u = A.work ? next_unit(A.work, lane) : blockIdx.x * kWarpsPerBlock + w;
    while (u < nunits) {
        prefix_item<D>(u, A, lane);
        if (!A.work) break;
        u = next_unit(A.work, lane);
    }
}

template <int NB, int D, bool XD>
__global__ void __launch_bounds__(32 * wpb<NB>(), kMinBlocks * kWarpsPerBlock / wpb<NB>()) k_seg_replay(RasterArgs A)
{
    constexpr int WPB = wpb<NB>();
    __shared__ float4 sr0[WPB][32 * NB], sr1[WPB][32 * NB], sr2[WPB][32 * NB];
    __shared__ uint32_t spos[WPB][32 * NB];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nunits = units_of(A, true);
    int u = A.work ? next_unit(A.work, lane) : blockIdx.x * WPB + w;
    while (u < nunits) {
        replay_item<NB, D, XD>(u, A, sr0[w], sr1[w], sr2[w], spos[w], lane);
        if (!A.work) break;
        u = next_unit(A.work, lane);
    }
}

template <int D>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, kMinBlocks) k_seg_finish(RasterArgs A, RasterOut O)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nunits = units_of(A, true);
    int u = A.work ? next_unit(A.work, lane) : blockIdx.x * kWarpsPerBlock + w;
    while (u < nunits) {
        finish_item<D>(u, A, O, lane);
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

// Sum 9 per-lane values over the warp: values 0..7 by a transposed butterfly
// (on return lane l holds the total of value l >> 2), value 8 by a plain one
// (*t8 in every lane) -- 14 shuffles where the 16-slot fold takes 16.
__device__ __forceinline__ float warp_transpose_reduce8(const float (&v)[16], float* t8)
{
    const unsigned lane = threadIdx.x & 31u;
    float w[4];
    {
        const bool up = lane & 16u;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float send = up ? v[k] : v[k + 4];
            const float keep = up ? v[k + 4] : v[k];
            w[k] = keep + __shfl_xor_sync(kFull, send, 16);
        }
    }
    {
        const bool up = lane & 8u;
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const float send = up ? w[k] : w[k + 2];
            const float keep = up ? w[k + 2] : w[k];
            w[k] = keep + __shfl_xor_sync(kFull, send, 8);
        }
    }
    {
        const bool up = lane & 4u;
        const float send = up ? w[0] : w[1];
        const float keep = up ? w[1] : w[0];
        w[0] = keep + __shfl_xor_sync(kFull, send, 4);
    }
    w[0] += __shfl_xor_sync(kFull, w[0], 2);
    w[0] += __shfl_xor_sync(kFull, w[0], 1);
    float x = v[8];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(kFull, x, off);
    *t8 = x;
    return w[0];
}

template <bool EXTRA, int NB, int D, bool DET>
__device__ __forceinline__ void bwd_item(int u, const RasterArgs& A, const RasterGrad& G, float4* sr0,
                                         float4* sr1, float4* sr2, uint32_t* spos, uint32_t* sg, int lane)
{
    Unit U;
    unit_of<D>(u, A, U);
    const LanePix<D> L(U, A.TS, lane);
    const unsigned lt = (1u << lane) - 1u;
    float T[D], R0[D], R1[D], R2[D], RD[D], RO[D], g0[D], g1[D], g2[D], gD[D], gO[D];
    uint32_t last[D];
    uint32_t wmax = 0;
#pragma unroll
    for (int j = 0; j < D; j++) {
        T[j] = 1.0f; R0[j] = R1[j] = R2[j] = RD[j] = RO[j] = 0.0f;
        g0[j] = g1[j] = g2[j] = gD[j] = gO[j] = 0.0f;
        last[j] = 0;
        if (L.inside[j]) {
            const size_t p = L.pix(U, j);
            last[j] = G.ncon[p];
            if (U.nseg == 1) {
                T[j] = G.Tfin[p];
            } else {
                const float* S = A.segstate;
                const int q = L.p[j];
                T[j] = S[seg_at(U.w, 0, q, A.TS)];
                R0[j] = S[seg_at(U.w, 1, q, A.TS)];
                R1[j] = S[seg_at(U.w, 2, q, A.TS)];
                R2[j] = S[seg_at(U.w, 3, q, A.TS)];
                RD[j] = S[seg_at(U.w, 4, q, A.TS)];
                RO[j] = S[seg_at(U.w, 5, q, A.TS)];
            }
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
    // positions at or beyond the last contributor reach no pixel of the block
    const uint32_t end = min(U.re, U.trs + wmax);
    if (end <= U.rs) return;
    // batches from the back: [bstart, bstart + 32 NB) with bstart = end - 32 NB k, clipped at rs
    constexpr int BS = 32 * NB;
    constexpr int PF = pf_slots<NB>();
    int64_t bstart = (int64_t)end - BS;
    float4 n0[PF], n1[PF], n2[PF], n3[PF];
    uint32_t ng[PF];
#pragma unroll
    for (int b = 0; b < PF; b++) {
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
            const int sl = PF == NB ? b : 0;
            const float4 c0 = n0[sl], c1 = n1[sl], c2 = n2[sl], c3 = n3[sl];
            const uint32_t cg = ng[sl];
            const int64_t i = bstart + b * 32 + lane;
            // next: the same sub-batch of the batch before (whole-batch
            // prefetch), else the next sub-batch of this one, or the first
            // of the batch before
            const int64_t ni = PF == NB ? i - BS : (b < NB - 1 ? i + 32 : i + 32 - 2 * BS);
            if (ni >= (int64_t)U.rs) {
                n0[sl] = A.s0[ni]; n1[sl] = A.s1[ni]; n2[sl] = A.s2[ni]; n3[sl] = A.s3[ni];
                ng[sl] = DET ? G.sinst[ni] : A.sgid[ni];
            }
            const bool hit = i >= (int64_t)U.rs && box_hit(c3, L.bx0, L.bx1, L.by0, L.by1);
            const unsigned mask = __ballot_sync(kFull, hit);
            if (hit) {
                const int k = nh + __popc(mask & lt);
                sr0[k] = c0; sr1[k] = c1; sr2[k] = c2;
                spos[k] = (uint32_t)(i - U.trs);
                sg[k] = cg;
            }
            nh += __popc(mask);
        }
        __syncwarp();
        for (int k = nh - 1; k >= 0; k--) {
            const float4 a = sr0[k], b = sr1[k], c = sr2[k];
            const uint32_t pos = spos[k];
            // Branch-free: a pixel the hit does not reach takes alpha = 0,
            // which leaves its R exactly unchanged (0 c + 1 R) and zeroes its
            // sums; only T needs a select.  No per-hit zeroing of the sums and
            // no divergent branch around the update.
            float v[16];
            bool any = false;
#pragma unroll
            for (int j = 0; j < D; j++) {
                float dx, dy, alpha;
                bool capped;
                const bool live = pair_eval_nb(a, b, L.px, L.py[j], dx, dy, alpha, capped) && pos < last[j];
                const float al = live ? alpha : 0.0f;
                T[j] = live ? __fdividef(T[j], 1.0f - al) : T[j];
                const float wgt = al * T[j];
                const float d0 = c.x - R0[j], d1 = c.y - R1[j], d2 = c.z - R2[j];
                float dot = g0[j] * d0 + g1[j] * d1 + g2[j] * d2;
                float dD = 0.0f, dO = 0.0f;
                if (EXTRA) {
                    dD = b.z - RD[j];
                    dO = 1.0f - RO[j];
                    dot += gD[j] * dD + gO[j] * dO;
                }
                // what is blended behind moves toward this Gaussian by alpha:
                // R + alpha (c - R) = alpha c + (1 - alpha) R
                R0[j] = fmaf(al, d0, R0[j]);
                R1[j] = fmaf(al, d1, R1[j]);
                R2[j] = fmaf(al, d2, R2[j]);
                if (EXTRA) {
                    RD[j] = fmaf(al, dD, RD[j]);
                    RO[j] = fmaf(al, dO, RO[j]);
                }
                // dL/d(exponent) = alpha dL/dalpha = alpha T g . (c - R)
                const float gp = capped ? 0.0f : wgt * dot;
                const float gx = gp * dx, gy = gp * dy;
                const float t[10] = {wgt * g0[j], wgt * g1[j], wgt * g2[j], gp, gx, gy, gx * dx, gx * dy, gy * dy,
                                     EXTRA ? wgt * gD[j] : 0.0f};
#pragma unroll
                for (int q = 0; q < 10; q++) v[q] = j == 0 ? t[q] : v[q] + t[q];
                any = any || live;
            }
#pragma unroll
            for (int q = 10; q < 16; q++) v[q] = 0.0f;
            if (__any_sync(kFull, any)) {
                if (EXTRA) {
                    const float r = warp_transpose_reduce16(v);
                    const int q = lane >> 1;
                    if ((lane & 1) == 0 && q < kNG) {
                        if (DET) G.part[((size_t)sg[k] * A.nblk + U.wb) * kNG + q] = r;
                        else atomicAdd(G.g2d + (size_t)sg[k] * kNG + q, r);
                    }
                } else {
                    // nine live slots (no depth or opacity gradient)
                    float r8;
                    const float r = warp_transpose_reduce8(v, &r8);
                    const int q = (lane & 3) == 0 ? (int)(lane >> 2) : (lane == 1 ? 8 : -1);
                    if (q >= 0) {
                        const float val = q == 8 ? r8 : r;
                        if (DET) G.part[((size_t)sg[k] * A.nblk + U.wb) * kNG + q] = val;
                        else atomicAdd(G.g2d + (size_t)sg[k] * kNG + q, val);
                    }
                }
            }
        }
        __syncwarp();
    }
}

template <bool EXTRA, int NB, int D, bool DET>
__global__ void __launch_bounds__(32 * wpb<NB>(), kMinBlocksBwd * kWarpsPerBlock / wpb<NB>())
k_raster_bwd(RasterArgs A, RasterGrad G)
{
    constexpr int WPB = wpb<NB>();
    __shared__ float4 sr0[WPB][32 * NB], sr1[WPB][32 * NB], sr2[WPB][32 * NB];
    __shared__ uint32_t spos[WPB][32 * NB], sg[WPB][32 * NB];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nunits = units_of(A, false);
    int u = A.work ? next_unit(A.work, lane) : blockIdx.x * WPB + w;
    while (u < nunits) {
        bwd_item<EXTRA, NB, D, DET>(u, A, G, sr0[w], sr1[w], sr2[w], spos[w], sg[w], lane);
        if (!A.work) break;
        u = next_unit(A.work, lane);
    }
}

// ---------------------------------------------------------------------------
// Per-Gaussian backward (Sec. III-D 1: threads assigned to the Gaussians
// rather than to the pixels).  A warp takes a (work item, 8x4 pixel block)
// unit like the kernel above and walks, back to front, the Gaussians whose
// alpha box touches the block (the hits); lane l owns hits l, l + 32, l + 64,
// ... and sums each one's gradient over the block's 32 pixels in its own
// registers.  The pixels' backward state -- the transmittance and the colour
// (depth, opacity) blended behind -- travels round the warp: at step s, lane
// l serves pixel p = (s - l) mod 32 for its hit s - p and then hands the
// pixel's state to lane l + 1, which holds the next hit.  Every pixel thus
// meets the hits in back-to-front order, one step apart, and H hits take
// H + 31 steps.  At step s lane s mod 32 is done with hit s - 32: it leaves
// its sums in a shared-memory slot and takes up hit s; every 32 steps the
// warp adds the 32 finished hits to their Gaussians' accumulators (or, in
// deterministic mode, stores them per instance and pixel block).  So a hit
// costs no warp reduction, and a Gaussian's sums stay in one lane.
// Hits are compacted from the sorted records in batches of 32, as above,
// into a per-warp ring of kPgQ entries, at least 32 ahead of the steps.  A
// list short enough to fit in the first fill (under 64 hits) is walked per
// pixel instead: there the 31 steps of filling and draining the ring would
// cost more than the per-hit reductions they save.
// ---------------------------------------------------------------------------
constexpr int kPgQ = 64;   // hit ring per warp: live hits are < 32 ahead + one batch of 32

struct PgWarp {
    float4 q0[kPgQ], q1[kPgQ], q2[kPgQ];   // hit records (sorted-order r0, r1, r2)
    uint32_t qpos[kPgQ], qg[kPgQ];          // list position (relative to the tile) and owner
    float4 pix[32];                         // per pixel: dL/dC and the last contributor (bits)
    float2 pxy[32];                         // per pixel: tile-relative coordinates
    float2 pde[32];                         // per pixel: dL/dD, dL/dO (EXTRA)
    float4 st0[32], st1[32];                // finished hits' sums, one slot per lane:
    float2 st2[32];                         //   0-3, 4-7, 8-9
    uint32_t stg[32];                       // their owners (0xffffffff: empty)
};
static_assert(sizeof(PgWarp) * 8 <= 48 * 1024, "static shared memory of the per-Gaussian backward");

template <bool EXTRA, bool DET>
__device__ __forceinline__ void pg_flush(const RasterArgs& A, const RasterGrad& G, int wb, uint32_t g,
                                         const float (&acc)[kNG])
{
    constexpr int NQ = EXTRA ? kNG : kNG - 1;
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        if (DET) G.part[((size_t)g * A.nblk + wb) * kNG + q] = acc[q];
        else atomicAdd(G.g2d + (size_t)g * kNG + q, acc[q]);
    }
}

template <bool EXTRA, bool DET>
__device__ __forceinline__ void bwd_item_pg(int u, const RasterArgs& A, const RasterGrad& G, PgWarp& W, int lane)
{
    Unit U;
    unit_of<1>(u, A, U);
    const unsigned lt = (1u << lane) - 1u;
    // lane l starts with the state of pixel (32 - l) mod 32 of the block
    const int p0 = (32 - lane) & 31;
    const int lx = U.lx0 + (p0 & 7), ly = U.ly0 + (p0 >> 3);
    const int x = U.x0 + (p0 & 7), y = U.y0 + (p0 >> 3);
    float T = 1.0f, R0 = 0.0f, R1 = 0.0f, R2 = 0.0f, RD = 0.0f, RO = 0.0f;
    uint32_t last = 0;
    float4 pc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float2 pe = make_float2(0.0f, 0.0f);
    if (x < U.W && y < U.H) {
        const size_t p = (size_t)U.pix_base + (size_t)y * U.W + x;
        last = G.ncon[p];
        if (U.nseg == 1) {
            T = G.Tfin[p];
        } else {
            const float* S = A.segstate;
            const int q = ly * A.TS + lx;
            T = S[seg_at(U.w, 0, q, A.TS)];
            R0 = S[seg_at(U.w, 1, q, A.TS)];
            R1 = S[seg_at(U.w, 2, q, A.TS)];
            R2 = S[seg_at(U.w, 3, q, A.TS)];
            RD = S[seg_at(U.w, 4, q, A.TS)];
            RO = S[seg_at(U.w, 5, q, A.TS)];
        }
        pc = make_float4(G.dL_drgb[3 * p], G.dL_drgb[3 * p + 1], G.dL_drgb[3 * p + 2], __uint_as_float(last));
        if (EXTRA) pe = make_float2(G.dL_ddepth ? G.dL_ddepth[p] : 0.0f, G.dL_dopac ? G.dL_dopac[p] : 0.0f);
    }
    W.pix[p0] = pc;
    W.pxy[p0] = make_float2((float)lx, (float)ly);
    if (EXTRA) W.pde[p0] = pe;
    W.stg[lane] = 0xffffffffu;
    uint32_t wmax = last;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wmax = max(wmax, __shfl_xor_sync(kFull, wmax, off));
    const uint32_t end = min(U.re, U.trs + wmax);
    __syncwarp();
    if (end <= U.rs) return;

    // batches from the back: [bstart, bstart + 32) clipped at rs, next one prefetched
    int64_t bstart = (int64_t)end - 32;
    float4 n0, n1, n2, n3;
    uint32_t ng = 0;
    {
        const int64_t i = bstart + lane;
        if (i >= (int64_t)U.rs) {
            n0 = A.s0[i]; n1 = A.s1[i]; n2 = A.s2[i]; n3 = A.s3[i];
            ng = DET ? G.sinst[i] : A.sgid[i];
        }
    }
    bool exhausted = false;
    int qhead = 0;   // hits compacted so far (hit 0 is the deepest)

    // the lane's current hit
    bool cur = false;
    float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = c0, c2 = c0;
    uint32_t cpos = 0, cg = 0;
    float acc[kNG];
#pragma unroll
    for (int q = 0; q < kNG; q++) acc[q] = 0.0f;

    for (int S = 0;; S += 32) {
        if (S > 0) {
            // the hits finished in the last 32 steps, one per lane
            const uint32_t g = W.stg[lane];
            if (g != 0xffffffffu) {
                float a[kNG];
                const float4 v0 = W.st0[lane], v1 = W.st1[lane];
                const float2 v2 = W.st2[lane];
                a[0] = v0.x; a[1] = v0.y; a[2] = v0.z; a[3] = v0.w;
                a[4] = v1.x; a[5] = v1.y; a[6] = v1.z; a[7] = v1.w;
                a[8] = v2.x; a[9] = v2.y;
                pg_flush<EXTRA, DET>(A, G, U.wb, g, a);
                W.stg[lane] = 0xffffffffu;
            }
        }
        // refill: compacted hits must cover the steps S .. S + 31
        while (!exhausted && qhead < S + 32) {
            const float4 b0 = n0, b1 = n1, b2 = n2, b3 = n3;
            const uint32_t bg = ng;
            const int64_t i = bstart + lane;
            const int64_t ni = i - 32;
            if (ni >= (int64_t)U.rs) {
                n0 = A.s0[ni]; n1 = A.s1[ni]; n2 = A.s2[ni]; n3 = A.s3[ni];
                ng = DET ? G.sinst[ni] : A.sgid[ni];
            }
            const bool hit = i >= (int64_t)U.rs && box_hit(b3, (float)U.x0, (float)(U.x0 + 7), (float)U.y0,
                                                            (float)(U.y0 + 3));
            const unsigned mask = __ballot_sync(kFull, hit);
            const int nh = __popc(mask);
            if (hit) {
                // deepest first: the batch's hits in reverse list order
                const int k = (qhead + nh - 1 - __popc(mask & lt)) & (kPgQ - 1);
                W.q0[k] = b0; W.q1[k] = b1; W.q2[k] = b2;
                W.qpos[k] = (uint32_t)(i - U.trs);
                W.qg[k] = bg;
            }
            qhead += nh;
            bstart -= 32;
            if (bstart + 32 <= (int64_t)U.rs) exhausted = true;
        }
        __syncwarp();
        if (S == 0 && exhausted) {
            // a short list (all of it fitted in the first fill): the ring
            // would spend 31 steps filling and draining for fewer than 64
            // hits, so walk it per pixel instead, each lane with the pixel
            // it holds, and fold each hit's sums across the warp
            const float px = (float)lx, py = (float)ly;
            for (int k = 0; k < qhead; k++) {
                const float4 a = W.q0[k], b = W.q1[k], c = W.q2[k];
                const uint32_t pos = W.qpos[k];
                float v[16];
#pragma unroll
                for (int q = 0; q < 16; q++) v[q] = 0.0f;
                float dx, dy, alpha;
                bool capped;
                const bool on = pos < last && pair_eval(a, b, px, py, dx, dy, alpha, capped);
                if (on) {
                    const float om = 1.0f - alpha;
                    T = __fdividef(T, om);
                    const float wgt = alpha * T;
                    float ga = pc.x * (c.x - R0) + pc.y * (c.y - R1) + pc.z * (c.z - R2);
                    if (EXTRA) ga += pe.x * (b.z - RD) + pe.y * (1.0f - RO);
                    ga *= T;
                    R0 = alpha * c.x + om * R0;
                    R1 = alpha * c.y + om * R1;
                    R2 = alpha * c.z + om * R2;
                    if (EXTRA) {
                        RD = alpha * b.z + om * RD;
                        RO = alpha + om * RO;
                    }
                    const float gp = capped ? 0.0f : ga * alpha;
                    v[0] = wgt * pc.x; v[1] = wgt * pc.y; v[2] = wgt * pc.z;
                    v[3] = gp;
                    v[4] = gp * dx; v[5] = gp * dy;
                    v[6] = gp * dx * dx; v[7] = gp * dx * dy; v[8] = gp * dy * dy;
                    if (EXTRA) v[9] = wgt * pe.x;
                }
                if (__any_sync(kFull, on)) {
                    const float r = warp_transpose_reduce16(v);
                    const int q = lane >> 1;
                    if ((lane & 1) == 0 && q < (EXTRA ? kNG : kNG - 1)) {
                        const uint32_t g = W.qg[k];
                        if (DET) G.part[((size_t)g * A.nblk + U.wb) * kNG + q] = r;
                        else atomicAdd(G.g2d + (size_t)g * kNG + q, r);
                    }
                }
            }
            __syncwarp();
            return;
        }
        if (exhausted && S > qhead + 30) break;
        // 32 steps of the wavefront
#pragma unroll 2
        for (int j = 0; j < 32; j++) {
            const int s = S + j;
            if (lane == j) {
                // done with hit s - 32: park its sums; take up hit s
                if (cur) {
                    W.st0[lane] = make_float4(acc[0], acc[1], acc[2], acc[3]);
                    W.st1[lane] = make_float4(acc[4], acc[5], acc[6], acc[7]);
                    W.st2[lane] = make_float2(acc[8], acc[9]);
                    W.stg[lane] = cg;
                }
                cur = s < qhead;
                if (cur) {
                    const int k = s & (kPgQ - 1);
                    c0 = W.q0[k]; c1 = W.q1[k]; c2 = W.q2[k];
                    cpos = W.qpos[k];
                    cg = W.qg[k];
                }
#pragma unroll
                for (int q = 0; q < kNG; q++) acc[q] = 0.0f;
            }
            const int p = (s - lane) & 31;
            const float4 c = W.pix[p];
            const float2 xy = W.pxy[p];
            float dx, dy, alpha;
            bool capped;
            if (cur && cpos < __float_as_uint(c.w) && pair_eval(c0, c1, xy.x, xy.y, dx, dy, alpha, capped)) {
                const float om = 1.0f - alpha;
                T = __fdividef(T, om);
                const float wgt = alpha * T;
                float ga = c.x * (c2.x - R0) + c.y * (c2.y - R1) + c.z * (c2.z - R2);
                float2 e = make_float2(0.0f, 0.0f);
                if (EXTRA) {
                    e = W.pde[p];
                    ga += e.x * (c1.z - RD) + e.y * (1.0f - RO);
                }
                ga *= T;
                R0 = alpha * c2.x + om * R0;
                R1 = alpha * c2.y + om * R1;
                R2 = alpha * c2.z + om * R2;
                if (EXTRA) {
                    RD = alpha * c1.z + om * RD;
                    RO = alpha + om * RO;
                }
                const float gp = capped ? 0.0f : ga * alpha;
                acc[0] += wgt * c.x; acc[1] += wgt * c.y; acc[2] += wgt * c.z;
                acc[3] += gp;
                acc[4] += gp * dx; acc[5] += gp * dy;
                acc[6] += gp * dx * dx; acc[7] += gp * dx * dy; acc[8] += gp * dy * dy;
                if (EXTRA) acc[9] += wgt * e.x;
            }
            // the pixel's state moves on to the lane of the next hit
            const int src = (lane + 31) & 31;
            T = __shfl_sync(kFull, T, src);
            R0 = __shfl_sync(kFull, R0, src);
            R1 = __shfl_sync(kFull, R1, src);
            R2 = __shfl_sync(kFull, R2, src);
            if (EXTRA) {
                RD = __shfl_sync(kFull, RD, src);
                RO = __shfl_sync(kFull, RO, src);
            }
        }
    }
    // the hits still held by the lanes
    if (cur) pg_flush<EXTRA, DET>(A, G, U.wb, cg, acc);
    __syncwarp();
}

template <bool EXTRA, bool DET>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, kMinBlocksBwd)
k_raster_bwd_pg(RasterArgs A, RasterGrad G)
{
    __shared__ PgWarp sw[kWarpsPerBlock];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nunits = units_of(A, false);
    int u = A.work ? next_unit(A.work, lane) : blockIdx.x * kWarpsPerBlock + w;
    while (u < nunits) {
        bwd_item_pg<EXTRA, DET>(u, A, G, sw[w], lane);
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

// Records in sorted-instance order (and the owning Gaussian of each), the
// mean made relative to the origin of the instance's tile: (u_hi - x0) is
// exact near the tile (Sterbenz), and adding u_lo leaves an offset accurate
// to float precision of a number of pixels, not of the image coordinate.
// The same pass marks each tile's list [first, last + 1) in `ranges` where
// the sorted tile id changes (tiles without instances keep the zeros the
// caller wrote).
__global__ void k_permute(const uint64_t* __restrict__ n_dev, uint32_t* __restrict__ ranges,
                          const uint32_t* __restrict__ sinst,
                          const uint32_t* __restrict__ stile, const ViewDesc* __restrict__ views, int V, int TS,
                          const uint32_t* __restrict__ owner, const float4* __restrict__ r0,
                          const float4* __restrict__ r1, const float4* __restrict__ r2,
                          const float4* __restrict__ r3, float4* __restrict__ s0, float4* __restrict__ s1,
                          float4* __restrict__ s2, float4* __restrict__ s3, uint32_t* __restrict__ sg)
{
    const uint64_t I = *n_dev;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < I; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t g = owner[sinst[i]];
        const int tile = (int)stile[i];
        if (i == 0 || stile[i - 1] != (uint32_t)tile) ranges[2 * tile] = (uint32_t)i;
        if (i == I - 1 || stile[i + 1] != (uint32_t)tile) ranges[2 * tile + 1] = (uint32_t)(i + 1);
        const ViewDesc& d = views[view_of_tile(views, V, tile)];
        const int lt = tile - d.tile_base;
        const float x0 = (float)((lt % d.TX) * TS), y0 = (float)((lt / d.TX) * TS);
        float4 a = r0[g];
        const float4 b = r1[g], c = r2[g];
        a.x = __fadd_rn(__fsub_rn(a.x, x0), c.w);
        a.y = __fadd_rn(__fsub_rn(a.y, y0), b.w);
        s0[i] = a; s1[i] = b; s2[i] = c; s3[i] = r3[g];
        sg[i] = g;
    }
}

// Resident CTAs of a kernel on the current device (SMs x CTAs per SM),
// looked up once per (kernel, device).
int resident_ctas(const void* kernel, int threads)
{
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({kernel, dev});
    if (it != cache.end()) return it->second;
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0);
    const int r = std::max(1, sm_count() * std::max(1, per));
    cache[{kernel, dev}] = r;
    return r;
}

// Grid of `wpb`-warp CTAs for up to units_bound warp units: one unit per
// warp, or (persistent) the resident CTAs, whose warps take units from a
// counter.
template <typename K>
int grid_for(K kernel, int64_t units_bound, bool persistent, int wpb = kWarpsPerBlock)
{
    const int64_t need = std::max<int64_t>(1, (units_bound + wpb - 1) / wpb);
    if (!persistent) return (int)std::min<int64_t>(need, 0x7fffffff);
    const int res = resident_ctas(reinterpret_cast<const void*>(kernel), 32 * wpb);
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, res));
}

int blocks_per_tile(const View& v) { return v.Ts * v.Ts / (32 * v.pd); }

// Split-tile items are bounded by 1.5 x capacity / seg: a tile of L >= 2 seg
// records has at most L / seg + 1 <= 1.5 L / seg segments.
int64_t split_items_bound(const View& v)
{
    return v.seg > 0 ? (int64_t)(v.itile.bytes / 4) * 3 / (2 * v.seg) + 1 : 0;
}

RasterArgs make_args(View& v, int* work)
{
    RasterArgs A;
    A.TS = v.Ts;
    A.V = v.V;
    A.nblk = blocks_per_tile(v);
    A.seg = v.seg;
    A.items = v.items.as<uint2>();
    A.ctl = v.count.as<uint64_t>();
    A.ranges = v.ranges.as<uint32_t>();
    A.s0 = v.srec0.as<float4>();
    A.s1 = v.srec1.as<float4>();
    A.s2 = v.srec2.as<float4>();
    A.s3 = v.srec3.as<float4>();
    A.sgid = v.sgid.as<uint32_t>();
    A.views = v.d_desc();
    A.segstate = v.segstate.as<float>();
    A.work = work;
    return A;
}

gl_status check_exec(const View& v)
{
    if (v.Ts != 8 && v.Ts != 16 && v.Ts != 32) { set_error("tile_size must be 8, 16 or 32"); return GL_ERR_INVALID; }
    if (v.nb != 1 && v.nb != 2 && v.nb != 4 && v.nb != 8) {
        set_error("batch depth must be 32, 64, 128 or 256");
        return GL_ERR_INVALID;
    }
    if (v.nb > 2 && v.pd != 1) {
        set_error("batch depths of 128 and 256 take one pixel per lane");
        return GL_ERR_INVALID;
    }
    if ((v.pd != 1 && v.pd != 2 && v.pd != 4) || 4 * v.pd > v.Ts) {
        set_error("pixels per lane must be 1, 2 or 4, with 4 x pixels per lane <= tile size");
        return GL_ERR_INVALID;
    }
    if (v.seg != 0 && (v.seg < 64 || v.seg > 65536 || (v.seg & (v.seg - 1)) != 0)) {
        set_error("segment length must be 0 or a power of two in 64..65536");
        return GL_ERR_INVALID;
    }
    return GL_OK;
}

template <int NB, int D, bool XD>
void fwd_launch(const RasterArgs& A, const RasterOut& O, int64_t units, int64_t split_units, bool persistent,
                int* work, cudaStream_t s)
{
    RasterArgs a1 = A;
    a1.work = work;
    k_raster_fwd<NB, D, XD><<<grid_for(k_raster_fwd<NB, D, XD>, units, persistent, wpb<NB>()), 32 * wpb<NB>(), 0,
                              s>>>(a1, O);
    if (split_units > 0) {
        // persistent grids take units from counters 2-4
        RasterArgs a2 = A, a3 = A, a4 = A;
        a2.work = work ? work + 2 : nullptr;
        a3.work = work ? work + 3 : nullptr;
        a4.work = work ? work + 4 : nullptr;
        k_seg_prefix<D><<<grid_for(k_seg_prefix<D>, split_units, persistent), 32 * kWarpsPerBlock, 0, s>>>(a2);
        k_seg_replay<NB, D, XD><<<grid_for(k_seg_replay<NB, D, XD>, split_units, persistent, wpb<NB>()),
                                  32 * wpb<NB>(), 0, s>>>(a3);
        k_seg_finish<D><<<grid_for(k_seg_finish<D>, split_units, persistent), 32 * kWarpsPerBlock, 0, s>>>(a4, O);
    }
}

template <bool EXTRA, int NB, int D, bool DET>
void bwd_launch(const RasterArgs& A, const RasterGrad& G, int64_t units, bool persistent, cudaStream_t s)
{
    const int grid = grid_for(k_raster_bwd<EXTRA, NB, D, DET>, units, persistent, wpb<NB>());
    k_raster_bwd<EXTRA, NB, D, DET><<<grid, 32 * wpb<NB>(), 0, s>>>(A, G);
}

template <bool EXTRA, bool DET>
void bwd_pg_launch(const RasterArgs& A, const RasterGrad& G, int64_t units, bool persistent, cudaStream_t s)
{
    const int grid = grid_for(k_raster_bwd_pg<EXTRA, DET>, units, persistent);
    k_raster_bwd_pg<EXTRA, DET><<<grid, 32 * kWarpsPerBlock, 0, s>>>(A, G);
}

template <bool EXTRA>
void bwd_dispatch(int nb, int pd, bool det, bool pg, const RasterArgs& A, const RasterGrad& G, int64_t units,
                  bool persistent, cudaStream_t s)
{
    if (pg) {    // per-Gaussian: batch depth 32, one pixel per lane
        if (det) bwd_pg_launch<EXTRA, true>(A, G, units, persistent, s);
        else bwd_pg_launch<EXTRA, false>(A, G, units, persistent, s);
    } else if (det) {   // batch depth 32 only
        if (pd == 1) bwd_launch<EXTRA, 1, 1, true>(A, G, units, persistent, s);
        else if (pd == 2) bwd_launch<EXTRA, 1, 2, true>(A, G, units, persistent, s);
        else bwd_launch<EXTRA, 1, 4, true>(A, G, units, persistent, s);
    } else if (nb == 4) {   // deeper batches: one pixel per lane
        bwd_launch<EXTRA, 4, 1, false>(A, G, units, persistent, s);
    } else if (nb == 8) {
        bwd_launch<EXTRA, 8, 1, false>(A, G, units, persistent, s);
    } else if (nb == 1) {
        if (pd == 1) bwd_launch<EXTRA, 1, 1, false>(A, G, units, persistent, s);
        else if (pd == 2) bwd_launch<EXTRA, 1, 2, false>(A, G, units, persistent, s);
        else bwd_launch<EXTRA, 1, 4, false>(A, G, units, persistent, s);
    } else {
        if (pd == 1) bwd_launch<EXTRA, 2, 1, false>(A, G, units, persistent, s);
        else if (pd == 2) bwd_launch<EXTRA, 2, 2, false>(A, G, units, persistent, s);
        else bwd_launch<EXTRA, 2, 4, false>(A, G, units, persistent, s);
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
    const int blocks = (int)std::min<size_t>(8 * (size_t)sm_count(), (I + 255) / 256);
    k_permute<<<blocks, 256, 0, s>>>(v.count.as<uint64_t>(), v.ranges.as<uint32_t>(), v.sorted_inst, v.sorted_tile, v.d_desc(), v.V, v.Ts,
                                     v.iowner.as<uint32_t>(),
                                     v.rec0.as<float4>(), v.rec1.as<float4>(), v.rec2.as<float4>(),
                                     v.rec3.as<float4>(), v.srec0.as<float4>(), v.srec1.as<float4>(),
                                     v.srec2.as<float4>(), v.srec3.as<float4>(), v.sgid.as<uint32_t>());
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

template <bool XD>
void fwd_dispatch(const View& v, const RasterArgs& A, const RasterOut& O, int64_t units, int64_t split_units,
                  int* work, cudaStream_t s)
{
    if (v.nb == 4) {
        fwd_launch<4, 1, XD>(A, O, units, split_units, v.persistent, work, s);
    } else if (v.nb == 8) {
        fwd_launch<8, 1, XD>(A, O, units, split_units, v.persistent, work, s);
    } else if (v.nb == 1) {
        if (v.pd == 1) fwd_launch<1, 1, XD>(A, O, units, split_units, v.persistent, work, s);
        else if (v.pd == 2) fwd_launch<1, 2, XD>(A, O, units, split_units, v.persistent, work, s);
        else fwd_launch<1, 4, XD>(A, O, units, split_units, v.persistent, work, s);
    } else {
        if (v.pd == 1) fwd_launch<2, 1, XD>(A, O, units, split_units, v.persistent, work, s);
        else if (v.pd == 2) fwd_launch<2, 2, XD>(A, O, units, split_units, v.persistent, work, s);
        else fwd_launch<2, 4, XD>(A, O, units, split_units, v.persistent, work, s);
    }
}

gl_status raster_forward(View& v, float* rgb, float* depth, float* opac, cudaStream_t s, bool extras)
{
    if (!extras && (depth || opac)) {
        set_error("raster_forward: depth and opacity outputs need the extra sums");
        return GL_ERR_INVALID;
    }
    const size_t P = (size_t)v.P;
    GL_TRY(v.Tfin.reserve(4 * P));
    GL_TRY(v.ncon.reserve(4 * P));
    if (v.ntiles == 0) return GL_OK;
    GL_TRY(check_exec(v));
    GL_TRY(v.work.reserve(32));
    const int64_t split = split_items_bound(v);
    if (split > 0) GL_TRY(v.segstate.reserve(sizeof(float) * kSegFields * (size_t)(v.Ts * v.Ts) * (size_t)split));
    PhaseScope ps(v.prof, PH_RASTER_FWD, s);
    int* work = nullptr;
    if (v.persistent) {
        work = v.work.as<int>();
        GL_CUDA_TRY(cudaMemsetAsync(work, 0, 8 * sizeof(int), s));
    }
    const RasterArgs A = make_args(v, nullptr);
    RasterOut O{rgb, depth, opac, v.Tfin.as<float>(), v.ncon.as<uint32_t>()};
    const int nblk = blocks_per_tile(v);
    const int64_t units = work_items_bound(v) * nblk, split_units = split * nblk;
    if (extras) fwd_dispatch<true>(v, A, O, units, split_units, work, s);
    else fwd_dispatch<false>(v, A, O, units, split_units, work, s);
    count_launches(split_units > 0 ? 4 : 1);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

gl_status raster_backward(View& v, const float* dL_drgb, const float* dL_ddepth,
                          const float* dL_dopac, cudaStream_t s)
{
    const size_t pairs = (size_t)v.n * v.V;
    GL_TRY(v.g2d.reserve(sizeof(float) * kNG * std::max<size_t>(pairs, 1)));
    GL_TRY(check_exec(v));
    GL_TRY(v.work.reserve(32));
    PhaseScope ps(v.prof, PH_RASTER_BWD, s);
    const bool det = v.det && v.ntiles > 0 && v.I != 0;
    // the per-Gaussian backward works on 8x4 pixel blocks whatever the
    // forward's pixels per lane
    const int nblk = v.pg ? v.Ts * v.Ts / 32 : blocks_per_tile(v);
    if (!det) GL_CUDA_TRY(cudaMemsetAsync(v.g2d.p, 0, sizeof(float) * kNG * pairs, s));
    if (v.ntiles == 0 || v.I == 0) return GL_OK;
    int* work = nullptr;
    if (v.persistent) {
        work = v.work.as<int>() + 1;
        GL_CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(int), s));
    }
    RasterArgs A = make_args(v, work);
    A.nblk = nblk;
    RasterGrad G{v.Tfin.as<float>(), v.ncon.as<uint32_t>(), dL_drgb, dL_ddepth, dL_dopac, v.g2d.as<float>(),
                 nullptr, v.sorted_inst};
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
    const int64_t units = work_items_bound(v) * nblk;
    if (dL_ddepth != nullptr || dL_dopac != nullptr)
        bwd_dispatch<true>(v.nb, v.pd, det, v.pg, A, G, units, v.persistent, s);
    else
        bwd_dispatch<false>(v.nb, v.pd, det, v.pg, A, G, units, v.persistent, s);
    count_launches(1);
    if (det) {
        const int blocks = (int)std::min<size_t>(8 * (size_t)sm_count(), (pairs + 255) / 256);
        k_part_reduce<<<std::max(blocks, 1), 256, 0, s>>>(v.gpart.as<float>(), v.touched.as<uint32_t>(),
                                                          v.dup_off.as<uint32_t>(), nblk, (int64_t)pairs,
                                                          v.count.as<uint64_t>(), (uint64_t)cap, v.g2d.as<float>());
        count_launches(1);
    }
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

}  // namespace gl
