// gl_binning.cu -- projection of every Gaussian (Eq. 1-3 and the SH colour)
// and tile binning: (tile | depth) ordering of the (Gaussian, tile) instances
// with a device LSD radix sort, then per-tile ranges (Sec. III-A, "sorting the
// Gaussians in depth order").
//
// Ordering strategy.  The instances must end up sorted by the 64-bit key
// (tile << 32 | float bits of depth), ties kept in emission order.  Instead of
// radix-sorting I 64-bit keys over 32 + log2(#tiles) bits, the Gaussians (N of
// them, N << I) are radix-sorted by depth first, instances are emitted in that
// order, and a stable radix sort on the tile id alone finishes the job.  The
// two give the same permutation: within a tile, stable order is depth order
// with ties broken by Gaussian index, which is the emission order of the
// single-key sort.
#include "gl_internal.h"

#include <algorithm>

namespace gl {

namespace {

constexpr int kPreThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kPreThreads * kScanItems;   // 1024 Gaussians per scan block
constexpr int kDupChunk = 4096;   // instances one duplication CTA writes at most

// Block-wide exclusive scan (NT threads); returns the exclusive prefix and
// writes the block total to *total.  `sm` needs NT/32 + 1 entries.
template <typename T, int NT>
__device__ __forceinline__ T block_exclusive_scan(T x, T* sm, T* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
    T incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sm[w] = incl;
    __syncthreads();
    if (w == 0) {
        T s = (lane < NW) ? sm[lane] : T(0);
        T si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(kFull, si, o);
            if (lane >= o) si += y;
        }
        if (lane < NW) sm[lane] = si - s;
        if (lane == NW - 1) sm[NW] = si;
    }
    __syncthreads();
    T res = sm[w] + incl - x;
    *total = sm[NW];
    __syncthreads();
    return res;
}

template <typename T, int NT>
__device__ __forceinline__ T block_sum(T x, T* sm)
{
    T tot;
    block_exclusive_scan<T, NT>(x, sm, &tot);
    return tot;
}

// ---------------------------------------------------------------------------
// K1: projection, colour and tile rectangle of every Gaussian.
// ---------------------------------------------------------------------------
template <int DEG>
__global__ void __launch_bounds__(kPreThreads)
k_preprocess(GParams p, const ViewDesc* __restrict__ views, int64_t total, int Ts, bool cull,
             float4* __restrict__ rec0, float4* __restrict__ rec1, float4* __restrict__ rec2,
             float4* __restrict__ rec3, int* __restrict__ radius, int4* __restrict__ rect,
             uint32_t* __restrict__ touched, uint32_t* __restrict__ dkey,
             unsigned long long* __restrict__ kmask, uint64_t* __restrict__ ctl)
{
    // t indexes (view, Gaussian) pairs: t = view * n + g
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t == 0) {
        ctl[2] = (uint64_t)total;   // keys of the depth sort
        ctl[3] = 0;
    }
    if (t >= total) return;
    const int vw = (int)(t / p.n);
    const int64_t g = t - (int64_t)vw * p.n;
    const Cam cam = views[vw].cam;
    const int TX = views[vw].TX, TY = views[vw].TY;
    constexpr int K = (DEG + 1) * (DEG + 1);
    float mu[3] = {p.means[3 * g], p.means[3 * g + 1], p.means[3 * g + 2]};
    float ls[3] = {p.log_scales[3 * g], p.log_scales[3 * g + 1], p.log_scales[3 * g + 2]};
    const float4 q4 = reinterpret_cast<const float4*>(p.quats)[g];
    float q[4] = {q4.x, q4.y, q4.z, q4.w};
    Decision D;
    if (!decide(mu, ls, q, p.logits[g], cam, Ts, TX, TY, D)) {
        radius[t] = 0;
        touched[t] = 0;
        dkey[t] = 0xffffffffu;
        rect[t] = make_int4(0, 0, 0, 0);
        return;
    }
    // raster records (not decisions): approximate reciprocal and logarithms,
    // a few ulp, far inside the pixels' tolerance and the alpha box's margin
    const float o = __fdividef(1.0f, 1.0f + __expf(-p.logits[g]));
    const float id = __fdividef(1.0f, D.det);
    // view direction from the camera centre c_w = -R^T t to the mean
    const float* R = cam.R;
    float cw0 = -(R[0] * cam.t[0] + R[3] * cam.t[1] + R[6] * cam.t[2]);
    float cw1 = -(R[1] * cam.t[0] + R[4] * cam.t[1] + R[7] * cam.t[2]);
    float cw2 = -(R[2] * cam.t[0] + R[5] * cam.t[1] + R[8] * cam.t[2]);
    float dx = mu[0] - cw0, dy = mu[1] - cw1, dz = mu[2] - cw2;
    float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    float Y[16];
    sh_eval<DEG>(dx * inv, dy * inv, dz * inv, Y);
    float c0 = 0.5f, c1 = 0.5f, c2 = 0.5f;
    const float* sh = p.sh + (size_t)g * K * 3;
    if ((K * 3) % 4 == 0) {
        const float4* s4 = reinterpret_cast<const float4*>(sh);
        float buf[K * 3];
#pragma unroll
        for (int i = 0; i < K * 3 / 4; i++) {
            float4 t = s4[i];
            buf[4 * i] = t.x; buf[4 * i + 1] = t.y; buf[4 * i + 2] = t.z; buf[4 * i + 3] = t.w;
        }
#pragma unroll
        for (int k = 0; k < K; k++) {
            c0 += Y[k] * buf[3 * k]; c1 += Y[k] * buf[3 * k + 1]; c2 += Y[k] * buf[3 * k + 2];
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; k++) {
            c0 += Y[k] * sh[3 * k]; c1 += Y[k] * sh[3 * k + 1]; c2 += Y[k] * sh[3 * k + 2];
        }
    }
    // log2-domain conic and opacity for the raster kernels
    const float A = D.c * id, B = -D.b * id, C = D.a * id;
    // the mean for rendering in double-float (hi in rec0, lo in rec2.w and
    // rec1.w); the permute makes it tile-relative
    float uh, ul, vh, vl;
    mean2d_df(mu, cam, uh, ul, vh, vl);
    rec0[t] = make_float4(uh, vh, -0.5f * kLog2e * A, -0.5f * kLog2e * C);
    rec1[t] = make_float4(-kLog2e * B, __log2f(o), D.z, vl);
    rec2[t] = make_float4(fmaxf(c0, 0.0f), fmaxf(c1, 0.0f), fmaxf(c2, 0.0f), ul);
    // conservative box of {alpha >= 1/255}: the ellipse d^T Sigma'^-1 d <= 2 ln(255 o)
    const float kappa = 2.0f * __logf(255.0f * o);
    if (kappa > 0.0f) {
        const float hx = sqrtf(kappa * D.a) * 1.001f + 0.01f, hy = sqrtf(kappa * D.c) * 1.001f + 0.01f;
        rec3[t] = make_float4(D.u - hx, D.u + hx, D.v - hy, D.v + hy);
    } else {
        rec3[t] = make_float4(3.0e38f, -3.0e38f, 3.0e38f, -3.0e38f);
    }
    radius[t] = D.r;
    rect[t] = make_int4(D.x0, D.y0, D.x1, D.y1);
    unsigned long long km;
    touched[t] = kept_tiles(D, Ts, cull, &km);
    dkey[t] = __float_as_uint(D.z);
    kmask[t] = km;
}

__global__ void k_set_u64(uint64_t* p, uint64_t v0, uint64_t v1)
{
    p[0] = v0;
    p[1] = v1;
}

// ---------------------------------------------------------------------------
// LSD radix sort of (u32 key, u32 value), 8-bit digits, stable.
//
// One histogram kernel counts the digits of every pass in a single read of
// the keys; then each pass is ONE scatter kernel over tiles of kOsTile keys.
// A CTA takes the next tile from a counter, ranks its keys by digit in
// shared memory, publishes the tile's per-digit counts and finds the counts
// of all earlier tiles by a chained scan with decoupled look-back (Merrill
// and Garland, "Single-pass Parallel Prefix Scan with Decoupled Look-back",
// 2016; the one-histogram-then-one-kernel-per-digit layout is the "Onesweep"
// sort of Adinets and Merrill, 2022).  Keys then leave the tile in digit
// order, so consecutive threads write consecutive addresses.  A pass whose
// digit is the same for every key (one non-empty histogram bin, seen on the
// device) copies its tiles through instead.
//
// Scratch (u32 words): global digit counts [pass][256] | tile counters
// [pass] | look-back words [pass][tiles][256], each (flag << 30 | count):
// flag 1 = this tile's count, flag 2 = inclusive count of tiles 0..t.
// A CTA only waits for tiles taken before its own, by CTAs already running,
// so the waits end; they are still bounded (kOsSpin polls), after which the
// CTA raises ctl[8] and goes on with the counts it has (its writes stay in
// bounds, the order is then wrong and the host reports GL_ERR_TIMEOUT).
// ---------------------------------------------------------------------------
constexpr int kOsThreads = 256;
constexpr int kOsItems = 15;
constexpr int kOsTile = kOsThreads * kOsItems;   // 3840 keys per tile
constexpr int kOsMaxPasses = 4;
constexpr int kOsTicketOff = kOsMaxPasses * 256;
constexpr int kOsStatusOff = kOsTicketOff + 64;
constexpr uint32_t kOsAgg = 1u << 30, kOsIncl = 2u << 30, kOsValMask = kOsAgg - 1u;
constexpr int kOsSpin = 1 << 20;   // polls of a tile not yet published before giving up
constexpr int kOsWindow = 16;      // earlier tiles read per look-back round trip

__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_gpu(uint32_t* p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Digit counts of all passes (scratch counts and counters zeroed before) and
// clearing of the look-back words of the tiles (tile_keys keys each) this
// sort visits.  A thread loads kOsHistKeys keys before counting any of them.
// With n_kept (zeroed before), keys 0xffffffff are left out of the counts and
// the number of the other keys is added to *n_kept.  For 32-bit keys the top
// digit takes few values (float keys of one range), so equal top digits of a
// warp are counted with one shared atomic.
constexpr int kOsHistKeys = 16;
__global__ void __launch_bounds__(kOsThreads)
k_os_hist(const uint32_t* __restrict__ kin, const uint64_t* n_dev, int passes, int tile_keys,
          int64_t tiles_max, uint32_t* __restrict__ scratch, unsigned long long* __restrict__ n_kept)
{
    __shared__ uint32_t h[kOsMaxPasses * 256];
    __shared__ unsigned long long s_kept;
    const uint64_t n = *n_dev;
    const bool drop = n_kept != nullptr;
    const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
    for (int i = threadIdx.x; i < kOsMaxPasses * 256; i += kOsThreads) h[i] = 0;
    if (threadIdx.x == 0) s_kept = 0;
    uint32_t kept = 0;
    const uint64_t nt = (n + tile_keys - 1) / tile_keys;
    const uint64_t gsz = (uint64_t)gridDim.x * kOsThreads;
    const uint64_t gid = (uint64_t)blockIdx.x * kOsThreads + threadIdx.x;
    uint32_t* status = scratch + kOsStatusOff;
    for (int p = 0; p < passes; p++)
        for (uint64_t i = gid; i < nt * 256; i += gsz) status[(uint64_t)p * tiles_max * 256 + i] = 0u;
    __syncthreads();
    // key j of a thread: b + (j / 4 * kOsThreads + threadIdx.x) * 4 + j % 4 (16-byte loads)
    for (uint64_t b = (uint64_t)blockIdx.x * kOsThreads * kOsHistKeys; b < n; b += gsz * kOsHistKeys) {
        uint32_t k[kOsHistKeys];
#pragma unroll
        for (int q = 0; q < kOsHistKeys / 4; q++) {
            const uint64_t i0 = b + ((uint64_t)q * kOsThreads + threadIdx.x) * 4;
            if (i0 + 3 < n) {
                const uint4 v = *reinterpret_cast<const uint4*>(kin + i0);
                k[4 * q] = v.x; k[4 * q + 1] = v.y; k[4 * q + 2] = v.z; k[4 * q + 3] = v.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; e++) k[4 * q + e] = i0 + e < n ? kin[i0 + e] : 0u;
            }
        }
#pragma unroll
        for (int j = 0; j < kOsHistKeys; j++) {
            const bool ok = b + ((uint64_t)(j / 4) * kOsThreads + threadIdx.x) * 4 + (j % 4) < n;
            const bool use = ok && !(drop && k[j] == 0xffffffffu);
            kept += use;
            if (passes == kOsMaxPasses) {   // uniform: every lane reaches the match
                if (use)
                    for (int p = 0; p < kOsMaxPasses - 1; p++) atomicAdd(&h[p * 256 + ((k[j] >> (8 * p)) & 255u)], 1u);
                const int dt = use ? (int)(k[j] >> 24) : -1;
                const unsigned peers = __match_any_sync(kFull, dt);
                if (use && (peers & lt) == 0) atomicAdd(&h[3 * 256 + dt], (uint32_t)__popc(peers));
            } else if (use) {
                for (int p = 0; p < passes; p++) atomicAdd(&h[p * 256 + ((k[j] >> (8 * p)) & 255u)], 1u);
            }
        }
    }
    if (drop) {
        for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(kFull, kept, o);
        if ((threadIdx.x & 31) == 0 && kept) atomicAdd(&s_kept, (unsigned long long)kept);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += kOsThreads)
        if (h[i]) atomicAdd(&scratch[i], h[i]);
    if (drop && threadIdx.x == 0 && s_kept) atomicAdd(n_kept, s_kept);
}

// One pass over tiles of NT x ITEMS keys (values 0, 1, 2, ... when vin is
// null; keys 0xffffffff left out when `drop`); threads 0..255 own one digit each
// in the per-digit phases (count, look-back, offsets).  Keys are ranked
// within a warp item by item: the lanes holding digit d set their bits in a
// shared mask word of d, read it back (the lanes below them with the same
// digit come first), and the lowest of them advances the warp's count of d
// and clears the mask.
template <int NT, int ITEMS, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_os_pass(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
          uint32_t* __restrict__ vout, const uint64_t* n_dev, int pass, int64_t tiles_max,
          uint32_t* __restrict__ scratch, unsigned long long* __restrict__ err, bool drop)
{
    static_assert(NT >= 256 && NT % 32 == 0, "a thread per digit");
    constexpr int TILE = NT * ITEMS;
    constexpr int NW = NT / 32;
    __shared__ uint32_t skey[TILE];
    __shared__ uint32_t sval[TILE];
    __shared__ uint32_t wcnt[NW][256];
    __shared__ uint32_t wmask[NW][256];
    __shared__ uint32_t dexcl[256];
    __shared__ uint32_t gbase[256];
    __shared__ uint32_t sm[NW + 1];
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const bool owner = tid < 256;
    const int shift = 8 * pass;
    const uint64_t n = *n_dev;
    const uint64_t nt = (n + TILE - 1) / TILE;
    if (tid == 0) s_tile = atomicAdd(&scratch[kOsTicketOff + pass], 1u);
    for (int d = lane; d < 256; d += 32) {
        wcnt[w][d] = 0u;
        wmask[w][d] = 0u;
    }
    // global digit offsets (while the tile counter answers)
    uint32_t tot;
    const uint32_t dcount = owner ? scratch[pass * 256 + tid] : 0u;
    const uint32_t gex = block_exclusive_scan<uint32_t, NT>(dcount, sm, &tot);
    // one digit holds every key: the stable pass keeps the order, so the
    // tile is copied through (no ranking, no look-back)
    const bool same = __syncthreads_or(n > 0 && (uint64_t)dcount == n);
    const uint32_t t = s_tile;
    if (t >= nt) return;
    const uint64_t base = (uint64_t)t * TILE;
    if (same) {
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
            const uint64_t idx = base + (uint64_t)j * NT + tid;
            if (idx < n) {
                kout[idx] = kin[idx];
                vout[idx] = vin ? vin[idx] : (uint32_t)idx;
            }
        }
        return;
    }
    const unsigned lt = (1u << lane) - 1u;

    // load (warp w holds the contiguous run [w * 32 * ITEMS, ...)) and rank
    // within the warp: earlier items, then lower lanes, come first;
    // rd[j] = rank within the warp's digit << 9 | digit (256: past the end)
    uint32_t kk[ITEMS], vv[ITEMS], rd[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        const uint64_t idx = base + (uint64_t)w * (32 * ITEMS) + j * 32 + lane;
        const bool ok = idx < n;
        kk[j] = ok ? kin[idx] : 0u;
        vv[j] = ok ? (vin ? vin[idx] : (uint32_t)idx) : 0u;
    }
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        const uint64_t idx = base + (uint64_t)w * (32 * ITEMS) + j * 32 + lane;
        const int d = (idx < n && !(drop && kk[j] == 0xffffffffu)) ? (int)((kk[j] >> shift) & 255u) : 256;
        if (d < 256) atomicOr(&wmask[w][d], 1u << lane);
        __syncwarp();
        const unsigned peers = d < 256 ? wmask[w][d] : 0u;
        const uint32_t prev = d < 256 ? wcnt[w][d] : 0u;
        rd[j] = ((prev + __popc(peers & lt)) << 9) | (uint32_t)d;
        __syncwarp();
        if (d < 256 && (peers & lt) == 0) {
            wcnt[w][d] = prev + __popc(peers);
            wmask[w][d] = 0u;
        }
        __syncwarp();
    }
    __syncthreads();

    // per digit: offsets of the warps, the tile's count, published at once
    uint32_t cnt = 0;
    uint32_t* status = scratch + kOsStatusOff + (uint64_t)pass * tiles_max * 256;
    uint32_t* mine = status + (uint64_t)t * 256 + tid;
    if (owner) {
#pragma unroll 8
        for (int ww = 0; ww < NW; ww++) {
            const uint32_t c = wcnt[ww][tid];
            wcnt[ww][tid] = cnt;
            cnt += c;
        }
        st_relaxed_gpu(mine, (t == 0 ? kOsIncl : kOsAgg) | cnt);
    }
    const uint32_t ex = block_exclusive_scan<uint32_t, NT>(owner ? cnt : 0u, sm, &tot);
    if (owner) dexcl[tid] = ex;
    __syncthreads();
    // the tile in digit order, in shared memory
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        const uint32_t d = rd[j] & 511u;
        if (d < 256) {
            const uint32_t pos = dexcl[d] + wcnt[w][d] + (rd[j] >> 9);
            skey[pos] = kk[j];
            sval[pos] = vv[j];
        }
    }

    // look back over the earlier tiles for this digit, kOsWindow of them per
    // round trip: add their counts in order up to the first inclusive one;
    // a tile not yet published ends the round (retried from there)
    uint32_t prefix = 0;
    if (owner && t > 0) {
        int64_t tt = (int64_t)t - 1;
        int spins = 0;
        while (true) {
            uint32_t sw[kOsWindow];
#pragma unroll
            for (int q = 0; q < kOsWindow; q++)
                sw[q] = tt - q >= 0 ? ld_relaxed_gpu(status + (uint64_t)(tt - q) * 256 + tid) : kOsIncl;
            uint32_t acc = 0;
            int used = 0, state = 0;   // 0: keep going, 1: inclusive count reached, 2: not yet published
#pragma unroll
            for (int q = 0; q < kOsWindow; q++) {
                if (state == 0) {
                    const uint32_t fl = sw[q] >> 30;
                    if (fl == 0) {
                        state = 2;
                    } else {
                        acc += sw[q] & kOsValMask;
                        used++;
                        if (fl == 2) state = 1;
                    }
                }
            }
            prefix += acc;
            tt -= used;
            if (state == 1) break;
            if (state == 2) {
                if (++spins >= kOsSpin) {
                    atomicOr(err, 1ull);
                    break;
                }
                __nanosleep(32);
            }
        }
        st_relaxed_gpu(mine, kOsIncl | (prefix + cnt));
    }
    if (owner) gbase[tid] = gex + prefix - ex;   // output index = gbase[d] + position in the digit-sorted tile
    __syncthreads();
    const int tn = (int)tot;   // the tile's keys that were ranked
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        const int i = tid + j * NT;
        if (i < tn) {
            const uint32_t k = skey[i];
            const uint64_t o = (uint64_t)(uint32_t)(gbase[(k >> shift) & 255u] + (uint32_t)i);
            if (o < n) {
                kout[o] = k;
                vout[o] = sval[i];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Scan of instance counts in depth order and duplication of the instances.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPreThreads)
k_scan_count(const uint32_t* __restrict__ sorted_g, const uint32_t* __restrict__ touched, const uint64_t* n_dev,
             uint64_t* __restrict__ bsum)
{
    const int64_t n = (int64_t)*n_dev;
    __shared__ uint64_t sm[kPreThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        int64_t j = base + k;
        if (j < n) s += touched[sorted_g[j]];
    }
    uint64_t tot = block_sum<uint64_t, kPreThreads>(s, sm);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Duplication parts of a scan block with x instances: one per kDupChunk of
// them, at least one.
__device__ __forceinline__ uint64_t dup_parts(uint64_t x)
{
    return x > (uint64_t)kDupChunk ? (x + kDupChunk - 1) / kDupChunk : 1ull;
}

// Exclusive scan of the block sums (bsum[0, nb)) and of the blocks'
// duplication parts (bsum[nb, 2 nb); count[10] = all parts).  count[3] =
// instances needed; if they fit in `cap` (and in 32 bits) count[0] = that
// number and count[1] = 0, else count[0] = 0 (nothing downstream runs) and
// count[1] = 1.
__global__ void __launch_bounds__(1024) k_scan_top(uint64_t* bsum, int nb, uint64_t cap,
                                                   uint64_t* count)
{
    __shared__ uint64_t sm[33];
    const int per = (nb + 1023) / 1024;
    const int b = min(nb, (int)threadIdx.x * per), e = min(nb, b + per);
    uint64_t s = 0, su = 0;
    for (int i = b; i < e; i++) {
        s += bsum[i];
        su += dup_parts(bsum[i]);
    }
    uint64_t tot, totu;
    uint64_t ex = block_exclusive_scan<uint64_t, 1024>(s, sm, &tot);
    uint64_t exu = block_exclusive_scan<uint64_t, 1024>(su, sm, &totu);
    uint64_t* uoff = bsum + nb;
    for (int i = b; i < e; i++) {
        uint64_t x = bsum[i];
        bsum[i] = ex;
        uoff[i] = exu;
        ex += x;
        exu += dup_parts(x);
    }
    if (threadIdx.x == 0) {
        count[10] = totu;
        const bool ovf = tot > cap || tot > 0xffffffffull;
        count[0] = ovf ? 0ull : tot;
        count[1] = ovf ? 1ull : 0ull;
        count[3] = tot;
    }
}

// Position of the n-th (0-based) set bit of m; m has more than n set bits.
// Halving search: at width w, skip the low w bits when they hold n or fewer.
__device__ __forceinline__ int nth_set_bit(unsigned long long m, int n)
{
    int pos = 0;
#pragma unroll
    for (int w = 32; w >= 1; w >>= 1) {
        const int c = __popcll(m & ((1ull << w) - 1ull));
        if (n >= c) {
            n -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// Emission of the instances.  The instances of consecutive Gaussians in
// depth order are consecutive, so a scan block's kScanBlock Gaussians own
// one contiguous output run.  The nearest Gaussians -- the first in depth
// order, the largest on screen -- cover the most tiles, so a run can be
// tens of times the average: it is cut into parts of kDupChunk outputs, one
// CTA each (the parts' offsets come from k_scan_top).  A CTA finds its
// block (a 32-way search over the part offsets by warp 0, one load round
// trip per level), reloads and scans the block's counts, and writes its
// part thread by thread (coalesced): output e belongs to the last Gaussian
// whose offset is <= e (binary search over the block's offsets in shared
// memory) and is its (e - offset)-th kept tile in row-major rectangle
// order.  A Gaussian's instances are written only if all of them fit in
// `cap`; the CTA holding its first output writes its offset.
static_assert(kScanBlock == 1024, "the emission search takes 10 halvings");

// Largest b < nb with off[b] <= e (off non-decreasing, off[0] = 0 <= e), in
// every lane of the calling warp.
__device__ __forceinline__ int find_block(const uint64_t* __restrict__ off, int nb, uint64_t e, int lane)
{
    int lo = 0, hi = nb;   // off[lo] <= e; the answer is in [lo, hi)
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) / 32;
        const int idx = lo + lane * step;
        const bool le = idx < hi && off[idx] <= e;
        const unsigned m = __ballot_sync(kFull, le);
        lo += (31 - __clz(m)) * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

__global__ void __launch_bounds__(kPreThreads)
k_duplicate(const uint32_t* __restrict__ sorted_g, const uint32_t* __restrict__ touched,
            const int4* __restrict__ rect, const uint64_t* __restrict__ bsum, int nb, const uint64_t* n_dev,
            const uint64_t* __restrict__ count, const ViewDesc* __restrict__ views, int64_t per_view, uint64_t cap,
            const unsigned long long* __restrict__ kmask,
            uint32_t* __restrict__ dup_off, uint32_t* __restrict__ itile, uint32_t* __restrict__ iowner)
{
    __shared__ uint64_t sm[kPreThreads / 32 + 1];
    __shared__ uint32_t s_off[kScanBlock + 1];   // run offsets in the scan block; [kScanBlock] = its total
    __shared__ uint32_t s_g[kScanBlock];
    __shared__ uint32_t s_t0[kScanBlock];        // tile of the rectangle's first cell
    __shared__ uint32_t s_wt[kScanBlock];        // rectangle width | tiles per row << 16
    __shared__ unsigned long long s_km[kScanBlock];
    __shared__ int s_b;
    const uint64_t part = blockIdx.x;
    if (part >= count[10]) return;
    const int64_t n = (int64_t)*n_dev;
    const uint64_t* uoff = bsum + nb;
    if (threadIdx.x < 32) {
        const int b = find_block(uoff, nb, part, threadIdx.x);
        if (threadIdx.x == 0) s_b = b;
    }
    __syncthreads();
    const int b = s_b;
    const uint64_t bbase = bsum[b];
    const int64_t base = (int64_t)b * kScanBlock + threadIdx.x * kScanItems;
    uint32_t gg[kScanItems], cc[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int64_t j = base + k;
        gg[k] = j < n ? sorted_g[j] : 0u;
        cc[k] = j < n ? touched[gg[k]] : 0u;
        s += cc[k];
    }
    uint64_t tot;
    uint64_t o = block_exclusive_scan<uint64_t, kPreThreads>(s, sm, &tot);
    // this CTA's part of the block's run
    const uint64_t r0 = (part - uoff[b]) * (uint64_t)kDupChunk;
    const uint64_t r1 = min(r0 + (uint64_t)kDupChunk, tot);
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int li = threadIdx.x * kScanItems + k;
        const uint32_t g = gg[k];
        s_off[li] = (uint32_t)o;
        s_g[li] = g;
        if (cc[k] && o < r1 && o + cc[k] > r0) {
            if (o >= r0) dup_off[g] = (uint32_t)(bbase + o);
            const int4 r = rect[g];
            const ViewDesc& vd = views[g / per_view];
            s_t0[li] = (uint32_t)(vd.tile_base + r.y * vd.TX + r.x);
            s_wt[li] = (uint32_t)(r.z - r.x) | ((uint32_t)vd.TX << 16);
            s_km[li] = kmask[g];
        }
        o += cc[k];
    }
    if (threadIdx.x == 0) s_off[kScanBlock] = (uint32_t)tot;
    __syncthreads();
    for (uint32_t e = (uint32_t)r0 + threadIdx.x; e < (uint32_t)r1; e += kPreThreads) {
        int lo = 0, hi = kScanBlock;   // s_off[lo] <= e < s_off[hi]
#pragma unroll
        for (int it = 0; it < 10; it++) {
            const int mid = (lo + hi) >> 1;
            if (s_off[mid] <= e) lo = mid; else hi = mid;
        }
        const uint32_t first = s_off[lo], cnt = s_off[lo + 1] - first;
        const uint64_t d = bbase + e;
        if (bbase + first + cnt > cap) continue;
        const uint32_t i = e - first;
        const unsigned long long km = s_km[lo];
        const int p = km == ~0ull ? (int)i : nth_set_bit(km, (int)i);
        const uint32_t wt = s_wt[lo];
        const uint32_t rw = wt & 0xffffu, TX = wt >> 16;
        itile[d] = s_t0[lo] + (uint32_t)(p / rw) * TX + (uint32_t)(p % rw);
        iowner[d] = s_g[lo];
    }
}

// Tile launch order: heaviest lists first (log2 buckets of the list length,
// longest-processing-time first), so long tiles start early instead of
// forming the tail.  Order within a bucket is arbitrary; tiles are
// independent, so results do not depend on it.
//
// Work items of the raster kernels, in tile launch order: one per tile, or,
// for a tile whose list holds at least 2 seg records, one per segment of
// seg records (seg a power of two, so such tiles sit in the log2 buckets
// ahead of all others and their items come first).  item = (tile,
// segment); count[6] = items, count[7] = items of split tiles.  One CTA of
// 1024 threads computes the tile launch order first, then the items.  With
// SMEM the list lengths and the order stay in shared memory (8 bytes per
// tile), so that the ranges are read once and nothing is read back.
constexpr int kOrderSmemTiles = 24576;   // 192 KB of shared memory
template <bool SMEM>
__global__ void __launch_bounds__(1024) k_order_items(const uint32_t* __restrict__ ranges, int ntiles, int seg,
                                                      uint32_t* __restrict__ order, uint2* __restrict__ items,
                                                      uint64_t* __restrict__ count)
{
    extern __shared__ uint32_t dyn[];   // SMEM: list length [ntiles] | order [ntiles]
    __shared__ uint32_t cnt[33], off[33];
    __shared__ uint32_t sm[1024 / 32 + 1];
    __shared__ uint32_t seg_end;
    uint32_t* slen = dyn;
    uint32_t* sord = dyn + ntiles;
    const uint2* r2 = reinterpret_cast<const uint2*>(ranges);
    if (threadIdx.x < 33) cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) seg_end = 0;
    __syncthreads();
    // bucket b = clz(length): 0 for the longest lists, 32 for empty ones
    constexpr int U = 4;   // lengths loaded before any is counted
    for (int t0 = threadIdx.x; t0 < ntiles; t0 += 1024 * U) {
        uint32_t L[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int t = t0 + u * 1024;
            L[u] = 0;
            if (t < ntiles) {
                const uint2 r = r2[t];
                L[u] = r.y - r.x;
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int t = t0 + u * 1024;
            if (t < ntiles) {
                if (SMEM) slen[t] = L[u];
                atomicAdd(&cnt[__clz(L[u])], 1u);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int b = 0; b < 33; b++) { off[b] = acc; acc += cnt[b]; }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += 1024) {
        uint32_t L;
        if (SMEM) {
            L = slen[t];
        } else {
            const uint2 r = r2[t];
            L = r.y - r.x;
        }
        const uint32_t pos = atomicAdd(&off[__clz(L)], 1u);
        order[pos] = (uint32_t)t;
        if (SMEM) sord[pos] = (uint32_t)t;
    }
    __syncthreads();   // the block's writes of order are visible to all its threads
    uint32_t carry = 0;
    for (int base = 0; base < ntiles; base += 1024) {
        const int k = base + threadIdx.x;
        uint32_t t = 0, nseg = 0;
        if (k < ntiles) {
            uint32_t L;
            if (SMEM) {
                t = sord[k];
                L = slen[t];
            } else {
                t = order[k];
                const uint2 r = r2[t];
                L = r.y - r.x;
            }
            nseg = (seg > 0 && L >= 2u * (uint32_t)seg) ? (L + seg - 1) / seg : 1u;
        }
        uint32_t tot;
        const uint32_t off0 = carry + block_exclusive_scan<uint32_t, 1024>(nseg, sm, &tot);
        for (uint32_t j = 0; j < nseg; j++) items[off0 + j] = make_uint2(t, j);
        if (nseg > 1) atomicMax(&seg_end, off0 + nseg);
        carry += tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        count[6] = carry;
        count[7] = seg_end;
    }
}

__global__ void k_export(const uint32_t* __restrict__ stile, const uint32_t* __restrict__ sinst,
                         const uint32_t* __restrict__ owner, const float4* __restrict__ rec1, int64_t I,
                         uint64_t* __restrict__ keys, uint32_t* __restrict__ vals)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < I; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t g = owner[sinst[i]];
        if (keys) keys[i] = ((uint64_t)stile[i] << 32) | (uint64_t)__float_as_uint(rec1[g].z);
        if (vals) vals[i] = g;
    }
}

// Projected quantities in plain form (mu', conic, opacity, rgb, depth).
__global__ void k_export_pre(const float4* __restrict__ rec0, const float4* __restrict__ rec1,
                             const float4* __restrict__ rec2, int64_t n, float* __restrict__ mean2d,
                             float* __restrict__ conic, float* __restrict__ opacity, float* __restrict__ rgb,
                             float* __restrict__ depth)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = rec0[g], b = rec1[g], c = rec2[g];
        if (mean2d) { mean2d[2 * g] = a.x; mean2d[2 * g + 1] = a.y; }
        if (conic) {
            conic[3 * g] = a.z / (-0.5f * kLog2e);
            conic[3 * g + 1] = b.x / -kLog2e;
            conic[3 * g + 2] = a.w / (-0.5f * kLog2e);
        }
        if (opacity) opacity[g] = exp2f(b.y);
        if (depth) depth[g] = b.z;
        if (rgb) { rgb[3 * g] = c.x; rgb[3 * g + 1] = c.y; rgb[3 * g + 2] = c.z; }
    }
}

__global__ void k_view_counts(const int* __restrict__ radius, int64_t n, const uint32_t* __restrict__ ncon,
                              int64_t P, unsigned long long* out)
{
    unsigned long long vis = 0, sc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) vis += radius[i] > 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += stride) sc += ncon[i];
    for (int off = 16; off > 0; off >>= 1) {
        vis += __shfl_xor_sync(kFull, vis, off);
        sc += __shfl_xor_sync(kFull, sc, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, vis);
        atomicAdd(out + 1, sc);
    }
}

__global__ void k_accumulate_counts(const int* __restrict__ radius, int64_t n, const uint32_t* __restrict__ ncon,
                                    int64_t P, const uint64_t* __restrict__ ctl, unsigned long long* acc)
{
    unsigned long long vis = 0, sc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) vis += radius[i] > 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += stride) sc += ncon[i];
    for (int off = 16; off > 0; off >>= 1) {
        vis += __shfl_xor_sync(kFull, vis, off);
        sc += __shfl_xor_sync(kFull, sc, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, vis);
        atomicAdd(acc + 2, sc);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(acc + 1, (unsigned long long)ctl[0]);
        atomicAdd(acc + 3, (unsigned long long)P);
    }
}

int ceil_log2(int64_t x)
{
    int b = 0;
    while ((int64_t(1) << b) < x) b++;
    return b;
}

}  // namespace

int64_t work_items_bound(const View& v)
{
    const int64_t cap = (int64_t)(v.itile.bytes / 4);
    return (int64_t)v.ntiles + (v.seg > 0 ? cap / v.seg + 1 : 0);
}

gl_status build_items(View& v, cudaStream_t s)
{
    GL_TRY(v.items.reserve(sizeof(uint2) * (size_t)std::max<int64_t>(work_items_bound(v), 1)));
    GL_TRY(v.tile_order.reserve(4 * (size_t)std::max(v.ntiles, 1)));
    if (v.ntiles <= kOrderSmemTiles) {
        const int bytes = 8 * std::max(v.ntiles, 1);
        GL_TRY(ensure_smem_limit(reinterpret_cast<const void*>(&k_order_items<true>), bytes));
        k_order_items<true><<<1, 1024, bytes, s>>>(v.ranges.as<uint32_t>(), v.ntiles, v.seg,
                                                   v.tile_order.as<uint32_t>(), v.items.as<uint2>(),
                                                   v.count.as<uint64_t>());
    } else {
        k_order_items<false><<<1, 1024, 0, s>>>(v.ranges.as<uint32_t>(), v.ntiles, v.seg,
                                                v.tile_order.as<uint32_t>(), v.items.as<uint2>(),
                                                v.count.as<uint64_t>());
    }
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

gl_status radix_sort_u32(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                         const uint64_t* n_dev, int64_t n_max, int64_t n_reserve, int bits, DevBuf& scratch,
                         uint64_t* ctl, uint32_t** out_k, uint32_t** out_v, cudaStream_t s, bool index_values,
                         uint64_t* n_kept)
{
    const int passes = std::max(1, std::min(kOsMaxPasses, (bits + 7) / 8));
    // look-back words sized for the larger of this sort and its reserve, so
    // that graph steps (whose bound is the capacity) never grow the buffer
    const int64_t nbig = std::max<int64_t>(std::max<int64_t>(n_max, n_reserve), 1);
    if (nbig >= (int64_t)kOsValMask) {
        set_error("radix sort: 2^30 keys or more");
        return GL_ERR_CAPACITY;
    }
    const int64_t tiles_max = (nbig + kOsTile - 1) / kOsTile;
    GL_TRY(scratch.reserve(sizeof(uint32_t) * ((size_t)kOsStatusOff + (size_t)kOsMaxPasses * tiles_max * 256)));
    uint32_t* sc = scratch.as<uint32_t>();
    GL_CUDA_TRY(cudaMemsetAsync(sc, 0, sizeof(uint32_t) * kOsStatusOff, s));
    const int tile_keys = kOsTile;
    const int64_t tiles = std::max<int64_t>(1, (n_max + tile_keys - 1) / tile_keys);
    const int hblocks = (int)std::min<int64_t>(
        4 * (int64_t)sm_count(), std::max<int64_t>(1, (n_max + kOsThreads * kOsHistKeys - 1) / (kOsThreads * kOsHistKeys)));
    unsigned long long* kept = reinterpret_cast<unsigned long long*>(n_kept);
    if (kept) GL_CUDA_TRY(cudaMemsetAsync(kept, 0, sizeof(uint64_t), s));
    k_os_hist<<<hblocks, kOsThreads, 0, s>>>(k0, n_dev, passes, tile_keys, tiles_max, sc, kept);
    uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
    unsigned long long* err = reinterpret_cast<unsigned long long*>(ctl + 8);
    for (int p = 0; p < passes; p++) {
        const uint32_t* vsrc = (p == 0 && index_values) ? nullptr : vi;
        // the first pass drops the 0xffffffff keys; the later ones sort the rest
        const uint64_t* np = (p > 0 && n_kept) ? n_kept : n_dev;
        k_os_pass<kOsThreads, kOsItems, 3><<<(unsigned)tiles, kOsThreads, 0, s>>>(ki, vsrc, ko, vo, np, p,
                                                                                  tiles_max, sc, err,
                                                                                  p == 0 && n_kept);
        std::swap(ki, ko);
        std::swap(vi, vo);
    }
    count_launches(1 + passes);
    GL_CUDA_TRY(cudaGetLastError());
    *out_k = ki;
    *out_v = vi;
    return GL_OK;
}

gl_status sort_wait_selftest(int32_t* expired)
{
    // two tiles of keys; the tile counter starts at 1, so the only CTA takes
    // tile 1 and looks back at tile 0, whose look-back words stay zero
    const uint64_t n = 2 * (uint64_t)kOsTile;
    const int64_t tiles_max = 2;
    const size_t words = (size_t)kOsStatusOff + (size_t)tiles_max * 256;
    struct Bufs {
        DevBuf keys, vals, kout, vout, scratch, ctl;
        ~Bufs()
        {
            for (DevBuf* b : {&keys, &vals, &kout, &vout, &scratch, &ctl}) b->release();
        }
    } B;
    DevBuf &keys = B.keys, &vals = B.vals, &kout = B.kout, &vout = B.vout, &scratch = B.scratch, &ctl = B.ctl;
    GL_TRY(keys.reserve(4 * n));
    GL_TRY(vals.reserve(4 * n));
    GL_TRY(kout.reserve(4 * n));
    GL_TRY(vout.reserve(4 * n));
    GL_TRY(scratch.reserve(4 * words));
    GL_TRY(ctl.reserve(16 * sizeof(uint64_t)));
    GL_CUDA_TRY(cudaMemset(keys.p, 0, 4 * n));
    GL_CUDA_TRY(cudaMemset(vals.p, 0, 4 * n));
    GL_CUDA_TRY(cudaMemset(scratch.p, 0, 4 * words));
    GL_CUDA_TRY(cudaMemset(ctl.p, 0, 16 * sizeof(uint64_t)));
    uint64_t* c = ctl.as<uint64_t>();
    GL_CUDA_TRY(cudaMemcpy(c, &n, sizeof(n), cudaMemcpyHostToDevice));   // ctl[0] = n
    const uint32_t one = 1;
    GL_CUDA_TRY(cudaMemcpy(scratch.as<uint32_t>() + kOsTicketOff, &one, sizeof(one), cudaMemcpyHostToDevice));
    k_os_pass<kOsThreads, kOsItems, 3><<<1, kOsThreads>>>(keys.as<uint32_t>(), vals.as<uint32_t>(), kout.as<uint32_t>(),
                                                         vout.as<uint32_t>(), c, 0, tiles_max, scratch.as<uint32_t>(),
                                                         reinterpret_cast<unsigned long long*>(c + 8), false);
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    GL_CUDA_TRY(cudaDeviceSynchronize());
    uint64_t flag = 0;
    GL_CUDA_TRY(cudaMemcpy(&flag, c + 8, sizeof(flag), cudaMemcpyDeviceToHost));
    *expired = flag ? 1 : 0;
    return GL_OK;
}

gl_status sort_wait_status(View& v, cudaStream_t s)
{
    if (!v.h_count || v.h_count[8] == 0) return GL_OK;
    GL_CUDA_TRY(cudaMemsetAsync(v.count.as<uint64_t>() + 8, 0, sizeof(uint64_t), s));
    set_error(v.h_count[8] & 2u ? "a bounded device wait gave up (parameter staging; the step's update is invalid)"
                                : "radix sort: a look-back wait gave up (result order invalid)");
    v.h_count[8] = 0;
    return GL_ERR_TIMEOUT;
}

gl_status accumulate_view_counts(const View& v, uint64_t* acc, cudaStream_t s)
{
    if (v.n * v.V == 0 && v.P == 0) return GL_OK;
    k_accumulate_counts<<<4 * sm_count(), 256, 0, s>>>(v.radius.as<int>(), v.n * v.V, v.ncon.as<uint32_t>(),
                                                      v.ncon.p ? v.P : 0, v.count.as<uint64_t>(),
                                                      reinterpret_cast<unsigned long long*>(acc));
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

gl_status view_counts(const View& v, int64_t* n_visible, int64_t* sum_contrib, cudaStream_t s)
{
    *n_visible = 0;
    *sum_contrib = 0;
    const int64_t P = v.P;
    if (v.n == 0 && P == 0) return GL_OK;
    unsigned long long* d = reinterpret_cast<unsigned long long*>(v.count.as<uint64_t>() + 4);
    GL_CUDA_TRY(cudaMemsetAsync(d, 0, 16, s));
    k_view_counts<<<4 * sm_count(), 256, 0, s>>>(v.radius.as<int>(), v.n * v.V, v.ncon.as<uint32_t>(), v.ncon.p ? P : 0, d);
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    unsigned long long h[2];
    GL_CUDA_TRY(cudaMemcpyAsync(h, d, 16, cudaMemcpyDeviceToHost, s));
    GL_CUDA_TRY(cudaStreamSynchronize(s));
    *n_visible = (int64_t)h[0];
    *sum_contrib = (int64_t)h[1];
    return GL_OK;
}

gl_status export_preprocess(const View& v, float* mean2d, float* conic, float* opacity, float* rgb,
                            float* depth, cudaStream_t s)
{
    if (v.n == 0) return GL_OK;
    int blocks = (int)std::min<int64_t>(4 * (int64_t)sm_count(), (v.n + 255) / 256);
    k_export_pre<<<blocks, 256, 0, s>>>(v.rec0.as<float4>(), v.rec1.as<float4>(), v.rec2.as<float4>(), v.n,
                                        mean2d, conic, opacity, rgb, depth);
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

gl_status export_instances(const View& v, uint64_t* keys, uint32_t* vals, cudaStream_t s)
{
    if (v.I == 0) return GL_OK;
    int blocks = (int)std::min<int64_t>(4 * (int64_t)sm_count(), (v.I + 255) / 256);
    k_export<<<blocks, 256, 0, s>>>(v.sorted_tile, v.sorted_inst, v.iowner.as<uint32_t>(),
                                    v.rec1.as<float4>(), v.I, keys, vals);
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

gl_status bin_view(View& v, const GParams& p, const Cam& cam, int Ts, cudaStream_t s)
{
    return bin_views(v, p, &cam, nullptr, 1, Ts, s);
}

void View::set_views(const Cam* cams, const ViewExtra* extra, int nv, int ts)
{
    V = nv;
    Ts = ts;
    W = cams[0].W;
    H = cams[0].H;
    TX = (cams[0].W + ts - 1) / ts;
    TY = (cams[0].H + ts - 1) / ts;
    cam = cams[0];
    int tiles = 0, ltiles = 0;
    int64_t pix = 0;
    for (int i = 0; i < nv; i++) {
        ViewDesc& d = hdesc[i];
        d = ViewDesc{};
        d.cam = cams[i];
        d.TX = (cams[i].W + ts - 1) / ts;
        d.TY = (cams[i].H + ts - 1) / ts;
        d.tile_base = tiles;
        d.ltile_base = ltiles;
        d.pix_base = pix;
        const ViewExtra ex = extra ? extra[i] : ViewExtra{};
        d.target = ex.target;
        d.E = ex.E;
        d.Em = ex.Em;
        d.e_bc1 = ex.e_bc1;
        d.e_bc2 = ex.e_bc2;
        d.weight = ex.weight;
        tiles += d.TX * d.TY;
        ltiles += ((cams[i].W + 31) / 32) * ((cams[i].H + 31) / 32);
        pix += (int64_t)cams[i].W * cams[i].H;
    }
    ntiles = tiles;
    nltiles = ltiles;
    P = pix;
}

gl_status bin_views(View& v, const GParams& p, const Cam* cams, const ViewExtra* extra, int V, int Ts,
                    cudaStream_t s, bool sync_free)
{
    if (V < 1 || V > kMaxViews) { set_error("1..64 views per step"); return GL_ERR_INVALID; }
    v.n = p.n;
    if (!sync_free) {
        v.set_views(cams, extra, V, Ts);
        GL_TRY(v.upload_descs(s));
    } else if (v.V != V || v.Ts != Ts) {
        set_error("view descriptors not set for this step");
        return GL_ERR_INVALID;
    }

    const ViewDesc* dv = v.d_desc();
    const int64_t n = p.n * V;   // (view, Gaussian) pairs
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    GL_TRY(v.rec0.reserve(16 * nn));
    GL_TRY(v.rec1.reserve(16 * nn));
    GL_TRY(v.rec2.reserve(16 * nn));
    GL_TRY(v.rec3.reserve(16 * nn));
    GL_TRY(v.radius.reserve(4 * nn));
    GL_TRY(v.rect.reserve(16 * nn));
    GL_TRY(v.touched.reserve(4 * nn));
    GL_TRY(v.dkey.reserve(4 * nn));
    GL_TRY(v.gidx.reserve(4 * nn));
    GL_TRY(v.dkey2.reserve(4 * nn));
    GL_TRY(v.gidx2.reserve(4 * nn));
    GL_TRY(v.dup_off.reserve(4 * nn));
    GL_TRY(v.kmask.reserve(8 * nn));
    const int nb = (int)((n + kScanBlock - 1) / kScanBlock);
    GL_TRY(v.bsum.reserve(16 * (size_t)std::max(nb, 1)));   // block offsets, then their duplication parts
    GL_TRY(v.ranges.reserve(8 * (size_t)v.ntiles));
    GL_CUDA_TRY(cudaMemsetAsync(v.ranges.p, 0, 8 * (size_t)v.ntiles, s));

    uint64_t* count = v.count.as<uint64_t>();
    if (n == 0) {
        v.I = 0;
        k_set_u64<<<1, 1, 0, s>>>(count, 0, 0);
        count_launches(1);
        GL_CUDA_TRY(cudaGetLastError());
        return build_items(v, s);
    }
    dim3 grid((unsigned)((n + kPreThreads - 1) / kPreThreads));
    {
    PhaseScope ps(v.prof, PH_PREPROCESS, s);
    count_launches(1);
    switch (p.deg) {
        case 0: k_preprocess<0><<<grid, kPreThreads, 0, s>>>(p, dv, n, Ts, v.cull, v.rec0.as<float4>(), v.rec1.as<float4>(), v.rec2.as<float4>(), v.rec3.as<float4>(), v.radius.as<int>(), v.rect.as<int4>(), v.touched.as<uint32_t>(), v.dkey.as<uint32_t>(), v.kmask.as<unsigned long long>(), count); break;
        case 1: k_preprocess<1><<<grid, kPreThreads, 0, s>>>(p, dv, n, Ts, v.cull, v.rec0.as<float4>(), v.rec1.as<float4>(), v.rec2.as<float4>(), v.rec3.as<float4>(), v.radius.as<int>(), v.rect.as<int4>(), v.touched.as<uint32_t>(), v.dkey.as<uint32_t>(), v.kmask.as<unsigned long long>(), count); break;
        case 2: k_preprocess<2><<<grid, kPreThreads, 0, s>>>(p, dv, n, Ts, v.cull, v.rec0.as<float4>(), v.rec1.as<float4>(), v.rec2.as<float4>(), v.rec3.as<float4>(), v.radius.as<int>(), v.rect.as<int4>(), v.touched.as<uint32_t>(), v.dkey.as<uint32_t>(), v.kmask.as<unsigned long long>(), count); break;
        case 3: k_preprocess<3><<<grid, kPreThreads, 0, s>>>(p, dv, n, Ts, v.cull, v.rec0.as<float4>(), v.rec1.as<float4>(), v.rec2.as<float4>(), v.rec3.as<float4>(), v.radius.as<int>(), v.rect.as<int4>(), v.touched.as<uint32_t>(), v.dkey.as<uint32_t>(), v.kmask.as<unsigned long long>(), count); break;
        default: set_error("sh_degree must be 0..3"); return GL_ERR_INVALID;
    }
    GL_CUDA_TRY(cudaGetLastError());
    }

    // depth order of the Gaussians; the culled ones (key 0xffffffff) are
    // dropped, count[9] = the Gaussians left
    uint32_t *sk, *sv;
    {
        PhaseScope ps(v.prof, PH_DEPTH_SORT, s);
        GL_TRY(radix_sort_u32(v.dkey.as<uint32_t>(), v.gidx.as<uint32_t>(), v.dkey2.as<uint32_t>(),
                              v.gidx2.as<uint32_t>(), count + 2, n, n, 32, v.hist, count, &sk, &sv, s,
                              true, count + 9));
    }
    v.sorted_g = sv;

    // instance offsets in depth order
    const uint64_t cap = v.itile.bytes / 4;
    if (sync_free && cap == 0) {
        set_error("graph steps need instance buffers sized by an earlier step");
        return GL_ERR_INVALID;
    }
    PhaseScope ps_scan(v.prof, PH_SCAN_DUP, s);
    k_scan_count<<<nb, kPreThreads, 0, s>>>(v.sorted_g, v.touched.as<uint32_t>(), count + 9, v.bsum.as<uint64_t>());
    k_scan_top<<<1, 1024, 0, s>>>(v.bsum.as<uint64_t>(), nb, cap, count);
    count_launches(2);
    GL_CUDA_TRY(cudaGetLastError());
    int64_t nmax;   // bound on the instance count the device holds in count[0]
    if (sync_free) {
        v.I = -1;   // known on the device only
        nmax = (int64_t)cap;
    } else {
        GL_CUDA_TRY(cudaMemcpyAsync(v.h_count, count, kCountCopy, cudaMemcpyDeviceToHost, s));
        GL_CUDA_TRY(cudaStreamSynchronize(s));
        GL_TRY(sort_wait_status(v, s));
        const uint64_t I = v.h_count[3];
        if (I > 0xffffffffull) {
            set_error("more than 2^32-1 (Gaussian, tile) instances in one step");
            return GL_ERR_CAPACITY;
        }
        v.I = (int64_t)I;
        if (I > cap) {
            // grow with headroom, so that later graph steps rarely overflow
            const size_t want = (size_t)(I + I / 4 + 1024);
            GL_TRY(v.itile.reserve(4 * want));
            GL_TRY(v.ival.reserve(4 * want));
            GL_TRY(v.itile2.reserve(4 * want));
            GL_TRY(v.ival2.reserve(4 * want));
            GL_TRY(v.iowner.reserve(4 * want));
            k_set_u64<<<1, 1, 0, s>>>(count, I, 0);
            count_launches(1);
        }
        nmax = (int64_t)I;
    }
    const uint64_t cap2 = v.itile.bytes / 4;
    // one CTA per duplication part: at most one per scan block plus one per
    // kDupChunk instances (their bound: the capacity for graph steps, else
    // the count just read)
    const int64_t nchunk = nb + (std::min<int64_t>(nmax, (int64_t)cap2) + kDupChunk - 1) / kDupChunk;
    k_duplicate<<<(unsigned)nchunk, kPreThreads, 0, s>>>(v.sorted_g, v.touched.as<uint32_t>(), v.rect.as<int4>(),
                                                         v.bsum.as<uint64_t>(), nb, count + 9, count, dv, p.n, cap2,
                                                         v.kmask.as<unsigned long long>(), v.dup_off.as<uint32_t>(),
                                                         v.itile.as<uint32_t>(), v.iowner.as<uint32_t>());
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    ps_scan.close();
    GL_TRY(v.tile_order.reserve(4 * (size_t)v.ntiles));
    if (nmax == 0) {
        v.sorted_tile = v.itile.as<uint32_t>();
        v.sorted_inst = v.ival.as<uint32_t>();
        return build_items(v, s);
    }
    // stable sort of the instances by tile id
    const int tbits = std::max(1, ceil_log2(v.ntiles));
    {
        PhaseScope ps(v.prof, PH_TILE_SORT, s);
        GL_TRY(radix_sort_u32(v.itile.as<uint32_t>(), v.ival.as<uint32_t>(), v.itile2.as<uint32_t>(),
                              v.ival2.as<uint32_t>(), count, nmax, (int64_t)cap2, tbits, v.hist, count, &sk, &sv,
                              s, true));
    }
    v.sorted_tile = sk;
    v.sorted_inst = sv;
    {
        PhaseScope ps(v.prof, PH_RANGES, s);
        // the sorted records (and the tile ranges, found in the same pass)
        // always get the full capacity, so that graph steps (which size
        // nothing) find room for any count that fits
        GL_TRY(permute_records(v, (int64_t)(v.itile.bytes / 4), s));
        GL_TRY(build_items(v, s));
    }
    // the counters reach the host at the caller's next synchronisation
    // (sort_wait_status); graph steps copy them at the end of the step
    if (!sync_free) GL_CUDA_TRY(cudaMemcpyAsync(v.h_count, count, kCountCopy, cudaMemcpyDeviceToHost, s));
    return GL_OK;
}

}  // namespace gl
