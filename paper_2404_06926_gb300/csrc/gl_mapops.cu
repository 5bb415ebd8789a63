// gl_mapops.cu -- map creation and expansion (Sec. III-C 1-2).
//
// Sky: N_s points uniform by area on the upper hemisphere of radius R about
// the world origin, drawn from a counter-based SplitMix64 stream (Steele, Lea
// and Flood, 2014: output i = mix(seed + (i+1) * golden gamma), top 24 bits as
// a uniform); each gets the distance to its nearest other sky point as its
// isotropic scale.  The nearest neighbour comes from a uniform grid: points
// are sorted by a 30-bit cell key with the library's radix sort, and each
// point searches shells of cells around its own (Chebyshev radius 1, 2, ...)
// until the best distance found is below the searched radius -- every point
// outside it is at least that far -- so the result is the exact minimum over
// all other points, with the same float arithmetic per pair as a brute-force
// scan.
//
// Expansion (Eq. 8): a point is kept if it lies in front of the camera and,
// when masking, lands inside the image on a pixel whose rendered opacity is
// below tau; kept points are compacted in input order and initialised as
// Gaussians: centre = point, SH DC from colour, opacity o_a, identity
// rotation, isotropic scale d/f.
#include "gl_internal.h"

#include <algorithm>
#include <cmath>

namespace gl {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 4;
constexpr int kBlock = kThreads * kItems;

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t i)
{
    return (double)(splitmix64_at(seed, i) >> 40) * (1.0 / 16777216.0);
}

__global__ void k_sky_points(float* __restrict__ means, int64_t n, double radius, uint64_t seed)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double zc = uniform01(seed, 2ull * (uint64_t)i);
    const double ph = 2.0 * 3.14159265358979323846 * uniform01(seed, 2ull * (uint64_t)i + 1ull);
    const double rr = sqrt(1.0 - zc * zc);
    means[3 * i] = (float)(radius * rr * cos(ph));
    means[3 * i + 1] = (float)(radius * rr * sin(ph));
    means[3 * i + 2] = (float)(radius * zc);
}

// Grid of the sky's nearest-neighbour search: cubic cells of side c over
// [-R, R] x [-R, R] x [0, R], at most 1024 per axis (10 bits each of a
// 30-bit key, x fastest, so the cells of a row are consecutive keys).
struct SkyGrid {
    float R, c, inv_c;
    int nx, nz;
};

__device__ __forceinline__ int sky_cell(float v, float lo, const SkyGrid& G, int n)
{
    const int i = (int)floorf(__fmul_rn(__fsub_rn(v, lo), G.inv_c));
    return min(max(i, 0), n - 1);
}

__global__ void k_sky_cells(const float* __restrict__ xyz, int64_t n, SkyGrid G, uint32_t* __restrict__ key,
                            uint32_t* __restrict__ idx, uint64_t* __restrict__ ctl)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) {
        ctl[0] = (uint64_t)n;   // keys of the sort
        ctl[8] = 0;             // its bounded-wait flag
    }
    if (i >= n) return;
    const int ix = sky_cell(xyz[3 * i], -G.R, G, G.nx);
    const int iy = sky_cell(xyz[3 * i + 1], -G.R, G, G.nx);
    const int iz = sky_cell(xyz[3 * i + 2], 0.0f, G, G.nz);
    key[i] = (uint32_t)ix | ((uint32_t)iy << 10) | ((uint32_t)iz << 20);
    idx[i] = (uint32_t)i;
}

// First position in the sorted keys [0, n) whose key is >= k.
__device__ __forceinline__ int64_t lower_key(const uint32_t* __restrict__ keys, int64_t n, uint32_t k)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Squared distance, explicitly rounded in a fixed order.
__device__ __forceinline__ float sq_dist(float3 a, float3 b)
{
    const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Minimum over the points of cells x0..x1 of row (iy, iz).
__device__ __forceinline__ void scan_row(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ idx,
                                         const float* __restrict__ xyz, int64_t n, int64_t self, float3 me,
                                         int x0, int x1, int iy, int iz, float& best)
{
    const uint32_t row = ((uint32_t)iy << 10) | ((uint32_t)iz << 20);
    for (int64_t j = lower_key(keys, n, row | (uint32_t)x0); j < n && keys[j] <= (row | (uint32_t)x1); j++) {
        const int64_t o = idx[j];
        if (o == self) continue;
        best = fminf(best, sq_dist(me, make_float3(xyz[3 * o], xyz[3 * o + 1], xyz[3 * o + 2])));
    }
}

__global__ void __launch_bounds__(kThreads)
k_sky_nn(const float* __restrict__ xyz, int64_t n, SkyGrid G, const uint32_t* __restrict__ keys,
         const uint32_t* __restrict__ idx, float* __restrict__ log_scales, float* __restrict__ quats,
         float* __restrict__ logits, float* __restrict__ sh, int K, float logit)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float3 me = make_float3(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]);
    const int ix = sky_cell(me.x, -G.R, G, G.nx), iy = sky_cell(me.y, -G.R, G, G.nx);
    const int iz = sky_cell(me.z, 0.0f, G, G.nz);
    float best = 3.0e38f;
    const int kmax = max(G.nx, G.nz);
    for (int k = 1; k <= kmax; k++) {
        // the shell at Chebyshev distance k around the point's cell (the
        // whole 3 x 3 x 3 block for k = 1)
        for (int dz = -k; dz <= k; dz++) {
            const int z = iz + dz;
            if (z < 0 || z >= G.nz) continue;
            for (int dy = -k; dy <= k; dy++) {
                const int y = iy + dy;
                if (y < 0 || y >= G.nx) continue;
                if (k == 1 || max(abs(dy), abs(dz)) == k) {
                    scan_row(keys, idx, xyz, n, i, me, max(ix - k, 0), min(ix + k, G.nx - 1), y, z, best);
                } else {
                    if (ix - k >= 0) scan_row(keys, idx, xyz, n, i, me, ix - k, ix - k, y, z, best);
                    if (ix + k < G.nx) scan_row(keys, idx, xyz, n, i, me, ix + k, ix + k, y, z, best);
                }
            }
        }
        // every point outside the searched block is at least k cell sides away
        const float reach = (float)k * G.c * (1.0f - 1e-5f);
        if (best <= reach * reach) break;
    }
    const float ls = 0.5f * logf(best);
    log_scales[3 * i] = ls; log_scales[3 * i + 1] = ls; log_scales[3 * i + 2] = ls;
    reinterpret_cast<float4*>(quats)[i] = make_float4(1.f, 0.f, 0.f, 0.f);
    logits[i] = logit;
    float* sp = sh + (size_t)i * K * 3;
    const float dc = (1.0f - 0.5f) / kSH0;   // white
    sp[0] = dc; sp[1] = dc; sp[2] = dc;
    for (int k = 3; k < K * 3; k++) sp[k] = 0.0f;
}

// Keep flags of Eq. 8 with the same explicitly rounded projection as binning.
__global__ void __launch_bounds__(kThreads)
k_expand_flags(const float* __restrict__ xyz, int64_t n, Cam cam, const float* __restrict__ opac,
               float tau, int use_mask, uint32_t* __restrict__ flag, float* __restrict__ depth,
               uint64_t* __restrict__ bsum)
{
    __shared__ uint64_t red[kThreads / 32];
    uint64_t cnt = 0;
    const int64_t base = (int64_t)blockIdx.x * kBlock + threadIdx.x * kItems;
    const float* R = cam.R;
    for (int k = 0; k < kItems; k++) {
        const int64_t i = base + k;
        if (i >= n) break;
        const float p0 = xyz[3 * i], p1 = xyz[3 * i + 1], p2 = xyz[3 * i + 2];
        const float x = far_(far_(far_(fmr(R[0], p0), fmr(R[1], p1)), fmr(R[2], p2)), cam.t[0]);
        const float y = far_(far_(far_(fmr(R[3], p0), fmr(R[4], p1)), fmr(R[5], p2)), cam.t[1]);
        const float z = far_(far_(far_(fmr(R[6], p0), fmr(R[7], p1)), fmr(R[8], p2)), cam.t[2]);
        depth[i] = z;
        uint32_t keep = z > kZNear ? 1u : 0u;
        if (keep && use_mask) {
            const float iz = fdr(1.0f, z);
            const float u = far_(fmr(cam.fx, fmr(x, iz)), cam.cx);
            const float v = far_(fmr(cam.fy, fmr(y, iz)), cam.cy);
            const float pu = floorf(far_(u, 0.5f)), pv = floorf(far_(v, 0.5f));
            keep = 0u;
            if (pu >= 0.0f && pu < (float)cam.W && pv >= 0.0f && pv < (float)cam.H) {
                const size_t pix = (size_t)pv * cam.W + (size_t)pu;
                keep = opac[pix] < tau ? 1u : 0u;
            }
        }
        flag[i] = keep;
        cnt += keep;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(kFull, cnt, off);
    if (lane == 0) red[w] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t s = 0;
        for (int ww = 0; ww < kThreads / 32; ww++) s += red[ww];
        bsum[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(1024) k_expand_scan(uint64_t* bsum, int nb, uint64_t* total)
{
    __shared__ uint64_t sm[1024];
    // small: nb <= 1024 * per; sequential per-thread segments then a block scan
    const int per = (nb + 1023) / 1024;
    const int b = min(nb, (int)threadIdx.x * per), e = min(nb, b + per);
    uint64_t s = 0;
    for (int i = b; i < e; i++) s += bsum[i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint64_t v = threadIdx.x >= off ? sm[threadIdx.x - off] : 0;
        __syncthreads();
        sm[threadIdx.x] += v;
        __syncthreads();
    }
    uint64_t ex = sm[threadIdx.x] - s;
    for (int i = b; i < e; i++) {
        uint64_t x = bsum[i];
        bsum[i] = ex;
        ex += x;
    }
    if (threadIdx.x == 1023) *total = sm[1023];
}

__global__ void __launch_bounds__(kThreads)
k_expand_emit(const float* __restrict__ xyz, const float* __restrict__ rgb, int64_t n,
              const uint32_t* __restrict__ flag, const float* __restrict__ depth,
              const uint64_t* __restrict__ bsum, float fx, float logit, int K, GMut dst,
              int64_t off0, int64_t cap)
{
    __shared__ uint64_t sm[kThreads];
    const int64_t base = (int64_t)blockIdx.x * kBlock + threadIdx.x * kItems;
    uint64_t c = 0;
    for (int k = 0; k < kItems; k++)
        if (base + k < n) c += flag[base + k];
    sm[threadIdx.x] = c;
    __syncthreads();
    for (int off = 1; off < kThreads; off <<= 1) {
        uint64_t v = threadIdx.x >= off ? sm[threadIdx.x - off] : 0;
        __syncthreads();
        sm[threadIdx.x] += v;
        __syncthreads();
    }
    uint64_t pos = bsum[blockIdx.x] + sm[threadIdx.x] - c;
    for (int k = 0; k < kItems; k++) {
        const int64_t i = base + k;
        if (i >= n) break;
        if (!flag[i]) continue;
        const int64_t g = off0 + (int64_t)pos++;
        if (g >= cap) continue;
        dst.means[3 * g] = xyz[3 * i];
        dst.means[3 * g + 1] = xyz[3 * i + 1];
        dst.means[3 * g + 2] = xyz[3 * i + 2];
        const float ls = logf(depth[i] / fx);
        dst.log_scales[3 * g] = ls; dst.log_scales[3 * g + 1] = ls; dst.log_scales[3 * g + 2] = ls;
        reinterpret_cast<float4*>(dst.quats)[g] = make_float4(1.f, 0.f, 0.f, 0.f);
        dst.logits[g] = logit;
        float* s = dst.sh + (size_t)g * K * 3;
        s[0] = (rgb[3 * i] - 0.5f) / kSH0;
        s[1] = (rgb[3 * i + 1] - 0.5f) / kSH0;
        s[2] = (rgb[3 * i + 2] - 0.5f) / kSH0;
        for (int k2 = 3; k2 < K * 3; k2++) s[k2] = 0.0f;
    }
}

}  // namespace

gl_status sky_create(float* means, float* log_scales, float* quats, float* logits, float* sh, int K,
                     int64_t n, double radius, uint64_t seed, float opacity, cudaStream_t s)
{
    if (n <= 0) return GL_OK;
    if (n >= ((int64_t)1 << 30)) { set_error("too many sky points"); return GL_ERR_INVALID; }
    const unsigned grid = (unsigned)((n + kThreads - 1) / kThreads);
    k_sky_points<<<grid, kThreads, 0, s>>>(means, n, radius, seed);
    // cells about twice the mean spacing of n points on the hemisphere's
    // 2 pi R^2, at most 1000 across
    SkyGrid G;
    G.R = (float)radius;
    G.c = (float)std::max(radius * std::sqrt(2.0 * 3.14159265358979323846 / (double)n), 2.0 * radius / 1000.0);
    G.inv_c = 1.0f / G.c;
    G.nx = (int)std::min(1024.0, std::floor(2.0 * radius / (double)G.c) + 1.0);
    G.nz = (int)std::min(1024.0, std::floor(radius / (double)G.c) + 1.0);
    struct Tmp {
        DevBuf keys, vals, keys2, vals2, scratch, ctl;
        ~Tmp()
        {
            for (DevBuf* b : {&keys, &vals, &keys2, &vals2, &scratch, &ctl}) b->release();
        }
    } T;
    const size_t nn = (size_t)n;
    GL_TRY(T.keys.reserve(4 * nn));
    GL_TRY(T.vals.reserve(4 * nn));
    GL_TRY(T.keys2.reserve(4 * nn));
    GL_TRY(T.vals2.reserve(4 * nn));
    GL_TRY(T.ctl.reserve(16 * sizeof(uint64_t)));
    uint64_t* ctl = T.ctl.as<uint64_t>();
    k_sky_cells<<<grid, kThreads, 0, s>>>(means, n, G, T.keys.as<uint32_t>(), T.vals.as<uint32_t>(), ctl);
    count_launches(2);
    GL_CUDA_TRY(cudaGetLastError());
    uint32_t *sk, *sv;
    GL_TRY(radix_sort_u32(T.keys.as<uint32_t>(), T.vals.as<uint32_t>(), T.keys2.as<uint32_t>(),
                          T.vals2.as<uint32_t>(), ctl, n, n, 30, T.scratch, ctl, &sk, &sv, s));
    const float logit = logf(opacity / (1.0f - opacity));
    k_sky_nn<<<grid, kThreads, 0, s>>>(means, n, G, sk, sv, log_scales, quats, logits, sh, K, logit);
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    // the temporary buffers are released on return: wait for the kernels
    uint64_t flag = 0;
    GL_CUDA_TRY(cudaMemcpyAsync(&flag, ctl + 8, sizeof(flag), cudaMemcpyDeviceToHost, s));
    GL_CUDA_TRY(cudaStreamSynchronize(s));
    if (flag) {
        set_error("sky creation: a radix-sort wait gave up");
        return GL_ERR_TIMEOUT;
    }
    return GL_OK;
}

gl_status expand_points(const float* xyz, const float* rgb, int64_t n, const Cam& cam,
                        const float* opacity_map, float tau, int use_mask, float opacity_fg, int K,
                        GMut dst, int64_t dst_offset, int64_t dst_cap, DevBuf& flags, DevBuf& scan,
                        int64_t* n_added, cudaStream_t s)
{
    // Two passes: count (the caller grows the map), then emit.  `dst` may be
    // null on the counting pass.
    const int nb = (int)((n + kBlock - 1) / kBlock);
    GL_TRY(flags.reserve(8 * (size_t)std::max<int64_t>(n, 1)));
    GL_TRY(scan.reserve(8 * (size_t)(nb + 2)));
    uint32_t* fl = flags.as<uint32_t>();
    float* depth = reinterpret_cast<float*>(fl + std::max<int64_t>(n, 1));
    uint64_t* bs = scan.as<uint64_t>();
    if (dst.means == nullptr) {
        k_expand_flags<<<nb, kThreads, 0, s>>>(xyz, n, cam, opacity_map, tau, use_mask, fl, depth, bs);
        k_expand_scan<<<1, 1024, 0, s>>>(bs, nb, bs + nb);
        count_launches(2);
        GL_CUDA_TRY(cudaGetLastError());
        uint64_t tot = 0;
        GL_CUDA_TRY(cudaMemcpyAsync(&tot, bs + nb, 8, cudaMemcpyDeviceToHost, s));
        GL_CUDA_TRY(cudaStreamSynchronize(s));
        *n_added = (int64_t)tot;
        return GL_OK;
    }
    const float logit = logf(opacity_fg / (1.0f - opacity_fg));
    k_expand_emit<<<nb, kThreads, 0, s>>>(xyz, rgb, n, fl, depth, bs, cam.fx, logit, K, dst, dst_offset,
                                          dst_cap);
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

}  // namespace gl
