// gl_mapops.cu -- map creation and expansion (Sec. III-C 1-2).
//
// Sky: N_s points uniform by area on the upper hemisphere of radius R about
// the world origin, drawn from a counter-based SplitMix64 stream (Steele, Lea
// and Flood, 2014: output i = mix(seed + (i+1) * golden gamma), top 24 bits as
// a uniform); each gets the distance to its nearest other sky point as its
// isotropic scale (brute force, tiled through shared memory).
//
// Expansion (Eq. 8): a point is kept if it lies in front of the camera and,
// when masking, lands inside the image on a pixel whose rendered opacity is
// below tau; kept points are compacted in input order and initialised as
// Gaussians: centre = point, SH DC from colour, opacity o_a, identity
// rotation, isotropic scale d/f.
#include "gl_internal.h"

#include <algorithm>

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

__global__ void __launch_bounds__(kThreads)
k_sky_init(const float* __restrict__ xyz, int64_t n, float* __restrict__ log_scales,
           float* __restrict__ quats, float* __restrict__ logits, float* __restrict__ sh, int K,
           float logit)
{
    __shared__ float3 tile[kThreads];
    const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    float3 me = make_float3(0.f, 0.f, 0.f);
    if (i < n) me = make_float3(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]);
    float best = 3.0e38f;
    for (int64_t base = 0; base < n; base += kThreads) {
        const int64_t j = base + threadIdx.x;
        __syncthreads();
        if (j < n) tile[threadIdx.x] = make_float3(xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2]);
        __syncthreads();
        const int cnt = (int)min((int64_t)kThreads, n - base);
        for (int k = 0; k < cnt; k++) {
            if (base + k == i) continue;
            const float dx = me.x - tile[k].x, dy = me.y - tile[k].y, dz = me.z - tile[k].z;
            best = fminf(best, dx * dx + dy * dy + dz * dz);
        }
    }
    if (i >= n) return;
    const float ls = 0.5f * logf(best);
    log_scales[3 * i] = ls; log_scales[3 * i + 1] = ls; log_scales[3 * i + 2] = ls;
    reinterpret_cast<float4*>(quats)[i] = make_float4(1.f, 0.f, 0.f, 0.f);
    logits[i] = logit;
    float* s = sh + (size_t)i * K * 3;
    const float dc = (1.0f - 0.5f) / kSH0;   // white
    s[0] = dc; s[1] = dc; s[2] = dc;
    for (int k = 3; k < K * 3; k++) s[k] = 0.0f;
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
    const unsigned grid = (unsigned)((n + kThreads - 1) / kThreads);
    k_sky_points<<<grid, kThreads, 0, s>>>(means, n, radius, seed);
    const float logit = logf(opacity / (1.0f - opacity));
    k_sky_init<<<grid, kThreads, 0, s>>>(means, n, log_scales, quats, logits, sh, K, logit);
    count_launches(2);
    GL_CUDA_TRY(cudaGetLastError());
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
