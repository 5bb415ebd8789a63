// gl_loss.cu -- exposure-compensated photometric loss (Eq. 9) and its adjoint.
//
// L = (1 - lambda) mean |E[C] - C_bar| + lambda (1 - mean SSIM(E[C], C_bar)),
// E[C] = A C + b with the 3x4 exposure [A | b] of the view (Sec. III-C 3).
// SSIM uses an 11x11 Gaussian window (sigma 1.5), zero padding, C1 = 0.01^2,
// C2 = 0.03^2 -- the D-SSIM of 3DGS the paper cites.
//
// One CTA per 32x32 output tile does everything in shared memory: it loads the
// exposed colour and the target over the tile plus a 10-pixel halo, blurs the
// five moment maps separably over a 5-pixel halo, forms the SSIM map and its
// partials w.r.t. (mu_x, E[x^2], E[xy]), blurs those back (the adjoint of a
// zero-padded symmetric correlation is the same correlation) and adds the
// channel's part of dL/dC = A^T dL/dE[C] in registers (the thread owning a
// pixel is the same in every channel, so dL/dC is written once, after the
// third channel, and never read back).  In every pass a thread slides the 11 taps along a
// run of 3-8 outputs held in registers, so each shared-memory value is read
// once per run rather than once per tap and output; the run lengths (and the
// split of the horizontal adjoint by map) are chosen so that each pass gives
// the CTA's 256 threads close to a whole number of rounds of equal items
// (728 = 2.8 x 256, 252, 504 = 2 x 252, 256).  The maps of later passes
// reuse the space of those consumed (65 KB, three CTAs per SM).  Per-CTA
// partial sums of |.|, SSIM and dL/dE are reduced afterwards in a fixed
// order, in double.
#include "gl_internal.h"

#include <algorithm>

namespace gl {

namespace {

constexpr int LT = 32;
constexpr int HW = 5;                 // window half width
constexpr int RA = LT + 4 * HW;       // 52
constexpr int RB = LT + 2 * HW;       // 42
constexpr int kThreads = 256;
constexpr int kNP = 14;               // partials per CTA: 12 dL/dE, sum|d|, sum SSIM
constexpr int HR = 3;                 // outputs per thread, horizontal moment pass (RB = 14 x 3)
constexpr int VR = 7;                 // outputs per thread, vertical moment pass (RB = 6 x 7)
constexpr int AHR = 8;                // outputs per item, horizontal adjoint pass (LT = 4 x 8)
constexpr int AVR = 4;                // outputs per thread, vertical adjoint pass (LT = 8 x 4)
static_assert(RB % HR == 0 && RB % VR == 0 && LT % AHR == 0 && LT % AVR == 0, "run lengths must tile the maps");
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

// x and y over the tile and halo (later the three SSIM partial maps), then
// the five moment maps (later the horizontally blurred partials)
constexpr size_t kSmemFloats = 2 * RA * RA + 5 * RA * RB;
static_assert(3 * RB * RB <= 2 * RA * RA && 3 * RB * LT <= 5 * RA * RB, "aliased maps must fit");

// One view passed by value (the stateless and allocation-free entry points).
struct LossOne {
    const float* rgb;
    const float* target;
    const float* E;
    float* dL;
    int W, H;
};

// Grid: one CTA per 32x32 loss tile over all views.  With `views` null the
// single view `one` is used; otherwise view, images, exposure and weight
// come from the descriptors and images are the concatenated ones.
__global__ void __launch_bounds__(kThreads, 3)
k_loss(LossOne one, const ViewDesc* __restrict__ views, int V, const float* __restrict__ rgb_all,
       float* __restrict__ dL_all, float lambda, float* __restrict__ part)
{
    const float* rgb = one.rgb;
    const float* target = one.target;
    const float* E = one.E;
    float* dL_drgb = one.dL;
    int W = one.W, H = one.H;
    float weight = 1.0f;
    int lt = blockIdx.x;
    if (views) {
        const int v = view_of_ltile(views, V, lt);
        const ViewDesc& d = views[v];
        lt -= d.ltile_base;
        rgb = rgb_all + 3 * d.pix_base;
        dL_drgb = dL_all + 3 * d.pix_base;
        target = d.target;
        E = d.E;
        W = d.cam.W;
        H = d.cam.H;
        weight = d.weight;
    }
    extern __shared__ float sm[];
    float* xs = sm;
    float* ys = xs + RA * RA;
    float* hm = ys + RA * RA;          // 5 maps, RA rows x RB cols
    float* gmap = xs;                  // 3 maps, RB x RB (reuses x, y after the horizontal pass)
    float* hg = hm;                    // 3 maps, RB rows x LT cols (reuses hm)
    __shared__ float wt[11];
    __shared__ float Es[12];
    __shared__ float red[kNP][kThreads / 32];
    const int tid = threadIdx.x;
    if (tid < 11) {
        float s = 0.0f;
        for (int k = 0; k < 11; k++) s += expf(-(float)((k - HW) * (k - HW)) / 4.5f);
        wt[tid] = expf(-(float)((tid - HW) * (tid - HW)) / 4.5f) / s;
    }
    if (tid < 12) Es[tid] = E ? E[tid] : ((tid % 5 == 0) ? 1.0f : 0.0f);
    __syncthreads();
    const int LTX = (W + LT - 1) / LT;
    const int ox = (lt % LTX) * LT, oy = (lt / LTX) * LT;
    const float invN = 1.0f / (3.0f * (float)W * (float)H);
    const float gS = -lambda * invN * weight;
    const float gL1 = (1.0f - lambda) * invN * weight;
    float l1acc = 0.0f, sacc = 0.0f;
    const int lane = tid & 31, wid = tid >> 5;

    // the adjoint pass gives every thread one run of AVR rows of one column,
    // the same in every channel: its pixels' dL/dC stays in registers
    static_assert(LT * (LT / AVR) == kThreads, "one adjoint run per thread");
    float dC[AVR][3];
#pragma unroll
    for (int o = 0; o < AVR; o++) dC[o][0] = dC[o][1] = dC[o][2] = 0.0f;
    for (int ch = 0; ch < 3; ch++) {
        // exposure gradient partials of this channel: sum g C_j (j < 3), sum g
        float pe[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        const float e0 = Es[4 * ch], e1 = Es[4 * ch + 1], e2 = Es[4 * ch + 2], e3 = Es[4 * ch + 3];
        for (int e = tid; e < RA * RA; e += kThreads) {
            const int gx = ox - 2 * HW + e % RA, gy = oy - 2 * HW + e / RA;
            float x = 0.0f, y = 0.0f;
            if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
                const size_t p = (size_t)gy * W + gx;
                x = e0 * rgb[3 * p] + e1 * rgb[3 * p + 1] + e2 * rgb[3 * p + 2] + e3;
                y = target[3 * p + ch];
            }
            xs[e] = x;
            ys[e] = y;
        }
        __syncthreads();
        // horizontal pass of the five moments: a thread slides the 11 taps
        // along a run of HR outputs of one row, loading each input once
        for (int e = tid; e < RA * (RB / HR); e += kThreads) {
            const int r = e / (RB / HR), c0 = (e % (RB / HR)) * HR;
            float xv[HR + 10], yv[HR + 10];
#pragma unroll
            for (int k = 0; k < HR + 10; k++) { xv[k] = xs[r * RA + c0 + k]; yv[k] = ys[r * RA + c0 + k]; }
#pragma unroll
            for (int o = 0; o < HR; o++) {
                float s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
#pragma unroll
                for (int k = 0; k < 11; k++) {
                    const float x = xv[o + k], y = yv[o + k], wk = wt[k];
                    s0 += wk * x; s1 += wk * y; s2 += wk * x * x; s3 += wk * y * y; s4 += wk * x * y;
                }
                const int i = r * RB + c0 + o;
                hm[i] = s0; hm[RA * RB + i] = s1; hm[2 * RA * RB + i] = s2;
                hm[3 * RA * RB + i] = s3; hm[4 * RA * RB + i] = s4;
            }
        }
        __syncthreads();
        // vertical pass, SSIM and its partials: a thread takes a run of VR
        // rows of one column, one moment map at a time
        for (int e = tid; e < RB * (RB / VR); e += kThreads) {
            const int c = e % RB, r0 = (e / RB) * VR;
            float mom[5][VR];
#pragma unroll
            for (int m = 0; m < 5; m++) {
                float col[VR + 10];
#pragma unroll
                for (int k = 0; k < VR + 10; k++) col[k] = hm[m * RA * RB + (r0 + k) * RB + c];
#pragma unroll
                for (int o = 0; o < VR; o++) {
                    float a = 0.0f;
#pragma unroll
                    for (int k = 0; k < 11; k++) a += wt[k] * col[o + k];
                    mom[m][o] = a;
                }
            }
#pragma unroll
            for (int o = 0; o < VR; o++) {
                const int r = r0 + o;
                const int gx = ox - HW + c, gy = oy - HW + r;
                float ga = 0.0f, gb = 0.0f, gc = 0.0f;
                if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
                    const float mx = mom[0][o], my = mom[1][o], exx = mom[2][o], eyy = mom[3][o], exy = mom[4][o];
                    const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
                    const float N1 = 2.f * mx * my + kC1, N2 = 2.f * sxy + kC2;
                    const float D1 = mx * mx + my * my + kC1, D2 = sxx + syy + kC2;
                    // one approximate reciprocal (a few ulp) serves S and both
                    // partials: 1/D1 = D2 iD, 1/D2 = D1 iD
                    const float iD = __fdividef(1.0f, D1 * D2);
                    const float S = N1 * N2 * iD;
                    if (r >= HW && r < HW + LT && c >= HW && c < HW + LT) sacc += S;
                    const float dN1 = N2 * iD, dN2 = N1 * iD, dD1 = -S * (D2 * iD), dD2 = -S * (D1 * iD);
                    const float dmx = dN1 * 2.f * my - dN2 * 2.f * my + dD1 * 2.f * mx - dD2 * 2.f * mx;
                    ga = gS * dmx;
                    gb = gS * dD2;
                    gc = gS * 2.f * dN2;
                }
                const int i = r * RB + c;
                gmap[i] = ga; gmap[RB * RB + i] = gb; gmap[2 * RB * RB + i] = gc;
            }
        }
        __syncthreads();
        // adjoint, horizontal: one item per (map, row, run of AHR outputs)
        for (int e = tid; e < 3 * RB * (LT / AHR); e += kThreads) {
            const int m = e / (RB * (LT / AHR)), rr = e % (RB * (LT / AHR));
            const int r = rr / (LT / AHR), c0 = (rr % (LT / AHR)) * AHR;
            float row[AHR + 10];
#pragma unroll
            for (int k = 0; k < AHR + 10; k++) row[k] = gmap[m * RB * RB + r * RB + c0 + k];
#pragma unroll
            for (int o = 0; o < AHR; o++) {
                float a = 0.0f;
#pragma unroll
                for (int k = 0; k < 11; k++) a += wt[k] * row[o + k];
                hg[m * RB * LT + r * LT + c0 + o] = a;
            }
        }
        __syncthreads();
        // adjoint, vertical, and dL/dE[C] of the tile's pixels: runs of AVR rows of a column
        for (int e = tid; e < LT * (LT / AVR); e += kThreads) {
            const int c = e % LT, r0 = (e / LT) * AVR;
            float acc[3][AVR];
#pragma unroll
            for (int m = 0; m < 3; m++) {
                float col[AVR + 10];
#pragma unroll
                for (int k = 0; k < AVR + 10; k++) col[k] = hg[m * RB * LT + (r0 + k) * LT + c];
#pragma unroll
                for (int o = 0; o < AVR; o++) {
                    float a = 0.0f;
#pragma unroll
                    for (int k = 0; k < 11; k++) a += wt[k] * col[o + k];
                    acc[m][o] = a;
                }
            }
            // dL/dE[C]_ch of the pixels (x, y read again: their shared copy
            // now holds the partial maps); dL/dC += A_ch^T dL/dE[C]_ch, by
            // the thread that owns the pixel in every channel
#pragma unroll
            for (int o = 0; o < AVR; o++) {
                const int r = r0 + o;
                const int gx = ox + c, gy = oy + r;
                if (gx < W && gy < H) {
                    const size_t p = (size_t)gy * W + gx;
                    const float c0 = rgb[3 * p], c1 = rgb[3 * p + 1], c2 = rgb[3 * p + 2];
                    const float x = e0 * c0 + e1 * c1 + e2 * c2 + e3, y = target[3 * p + ch];
                    const float d = x - y;
                    l1acc += fabsf(d);
                    const float g = acc[0][o] + 2.f * x * acc[1][o] + y * acc[2][o] +
                                    gL1 * (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f));
                    pe[0] += g * c0; pe[1] += g * c1; pe[2] += g * c2; pe[3] += g;
                    dC[o][0] = ch == 0 ? e0 * g : dC[o][0] + e0 * g;
                    dC[o][1] = ch == 0 ? e1 * g : dC[o][1] + e1 * g;
                    dC[o][2] = ch == 0 ? e2 * g : dC[o][2] + e2 * g;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; i++) {
            float v = pe[i];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
            if (lane == 0) red[4 * ch + i][wid] = v;
        }
        __syncthreads();
    }

    {
        const int c = tid % LT, r0 = (tid / LT) * AVR;
#pragma unroll
        for (int o = 0; o < AVR; o++) {
            const int gx = ox + c, gy = oy + r0 + o;
            if (gx < W && gy < H) {
                const size_t p = (size_t)gy * W + gx;
                dL_drgb[3 * p] = dC[o][0];
                dL_drgb[3 * p + 1] = dC[o][1];
                dL_drgb[3 * p + 2] = dC[o][2];
            }
        }
    }
    {
        const float vals[2] = {l1acc, sacc};
#pragma unroll
        for (int i = 0; i < 2; i++) {
            float v = vals[i];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
            if (lane == 0) red[12 + i][wid] = v;
        }
    }
    __syncthreads();
    if (tid < kNP) {
        float v = 0.0f;
        for (int ww = 0; ww < kThreads / 32; ww++) v += red[tid][ww];
        part[(size_t)blockIdx.x * kNP + tid] = v;
    }
}

// Sums the per-tile partials in a fixed order (double).  Single view (views
// null): block 0 over [0, nblk) -> loss_out, dE_out.  Views: block v over the
// view's loss tiles -> loss_v[v] (unweighted) and, if the view has Em, one
// Adam step of its exposure on the (already weighted) gradient.
constexpr int kRedBatch = 8;
__global__ void k_loss_final(const float* __restrict__ part, int nblk, int W, int H, float lambda,
                             float* __restrict__ loss_out, float* __restrict__ dE_out,
                             const ViewDesc* __restrict__ views, float* __restrict__ loss_v, float b1,
                             float b2, float eps, float lr, const uint64_t* __restrict__ abort)
{
    __shared__ double tot[kNP];
    int begin = 0;
    float* Ev = nullptr;
    float* Em = nullptr;
    float bc1 = 1.f, bc2 = 1.f;
    if (views) {
        const ViewDesc& d = views[blockIdx.x];
        begin = d.ltile_base;
        W = d.cam.W;
        H = d.cam.H;
        nblk = ((W + LT - 1) / LT) * ((H + LT - 1) / LT);
        Ev = d.E;
        Em = d.Em;
        bc1 = d.e_bc1;
        bc2 = d.e_bc2;
    }
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k < kNP) {
        // lane sums of partials lane, lane + 32, ... in that order; kRedBatch
        // loads in flight before they are added
        double acc = 0.0;
        for (int i0 = lane; i0 < nblk; i0 += 32 * kRedBatch) {
            float x[kRedBatch];
#pragma unroll
            for (int b = 0; b < kRedBatch; b++) {
                const int i = i0 + 32 * b;
                x[b] = i < nblk ? part[(size_t)(begin + i) * kNP + k] : 0.0f;
            }
#pragma unroll
            for (int b = 0; b < kRedBatch; b++)
                if (i0 + 32 * b < nblk) acc += x[b];
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
        if (lane == 0) tot[k] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double invN = 1.0 / (3.0 * (double)W * (double)H);
        const double L = (1.0 - lambda) * tot[12] * invN + lambda * (1.0 - tot[13] * invN);
        if (views) { if (loss_v) loss_v[blockIdx.x] = (float)L; }
        else if (loss_out) *loss_out = (float)L;
    }
    if (threadIdx.x < 12) {
        const int i = threadIdx.x;
        const float g = (float)tot[i];
        if (!views && dE_out) dE_out[i] = g;
        if (Ev && Em && !(abort && abort[1])) {
            const float m = b1 * Em[i] + (1.0f - b1) * g;
            const float v = b2 * Em[12 + i] + (1.0f - b2) * g * g;
            Em[i] = m;
            Em[12 + i] = v;
            Ev[i] -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
        }
    }
}

__global__ void k_apply_exposure(const float* __restrict__ src, float* __restrict__ dst, int64_t P,
                                 float e0, float e1, float e2, float e3, float e4, float e5, float e6,
                                 float e7, float e8, float e9, float e10, float e11)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        const float c0 = src[3 * p], c1 = src[3 * p + 1], c2 = src[3 * p + 2];
        dst[3 * p] = e0 * c0 + e1 * c1 + e2 * c2 + e3;
        dst[3 * p + 1] = e4 * c0 + e5 * c1 + e6 * c2 + e7;
        dst[3 * p + 2] = e8 * c0 + e9 * c1 + e10 * c2 + e11;
    }
}

}  // namespace

int loss_partials_needed(int W, int H)
{
    return ((W + LT - 1) / LT) * ((H + LT - 1) / LT) * kNP;
}

namespace {
gl_status loss_attr()
{
    return ensure_smem_limit(reinterpret_cast<const void*>(&k_loss), (int)(kSmemFloats * sizeof(float)));
}
}  // namespace

gl_status photometric_loss(const float* rgb, const float* target, const float* E, int W, int H,
                           float lambda, float* dL_drgb, float* part, float* loss_out, float* dE_out,
                           cudaStream_t s)
{
    GL_TRY(loss_attr());
    const int nblk = ((W + LT - 1) / LT) * ((H + LT - 1) / LT);
    LossOne one{rgb, target, E, dL_drgb, W, H};
    k_loss<<<nblk, kThreads, kSmemFloats * sizeof(float), s>>>(one, nullptr, 0, nullptr, nullptr, lambda, part);
    k_loss_final<<<1, 32 * kNP, 0, s>>>(part, nblk, W, H, lambda, loss_out, dE_out, nullptr, nullptr, 0.f, 0.f,
                                        0.f, 0.f, nullptr);
    count_launches(2);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

gl_status photometric_loss_views(const View& v, const float* rgb, float lambda, float* dL_drgb, float* part,
                                 float* loss_v, float b1, float b2, float eps, float lr, cudaStream_t s,
                                 const uint64_t* abort)
{
    GL_TRY(loss_attr());
    LossOne one{};
    k_loss<<<v.nltiles, kThreads, kSmemFloats * sizeof(float), s>>>(one, v.d_desc(), v.V, rgb, dL_drgb, lambda,
                                                                     part);
    k_loss_final<<<v.V, 32 * kNP, 0, s>>>(part, 0, 0, 0, lambda, nullptr, nullptr, v.d_desc(), loss_v, b1, b2, eps,
                                          lr, abort);
    count_launches(2);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

gl_status apply_exposure(const float* src, float* dst, const float E[12], int64_t P, cudaStream_t s)
{
    int blocks = (int)std::min<int64_t>(8 * (int64_t)sm_count(), (P + 255) / 256);
    if (blocks < 1) blocks = 1;
    k_apply_exposure<<<blocks, 256, 0, s>>>(src, dst, P, E[0], E[1], E[2], E[3], E[4], E[5], E[6], E[7],
                                            E[8], E[9], E[10], E[11]);
    count_launches(1);
    GL_CUDA_TRY(cudaGetLastError());
    return GL_OK;
}

}  // namespace gl
