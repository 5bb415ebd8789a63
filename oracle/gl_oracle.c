/*
 * gl_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, single-threaded CPU restatement of one optimisation iteration
 * of the Gaussian-LIC photo-realistic map (arXiv 2404.06926): projection,
 * SH colour, tile binning, front-to-back compositing, exposure-compensated
 * L1 + D-SSIM loss, the analytic backward to every Gaussian attribute, the
 * camera pose and the exposure, Adam, sky creation and map expansion.
 * Only tests/, the smoke check and the benchmark's CPU-baseline leg load it.
 *
 * Precision.  Every continuous value is computed in double.  The arithmetic
 * that decides an integer -- the cull, the screen radius, the tile rectangle
 * and the depth key -- is computed in float32 in a fixed operation order with
 * no contraction (build with -ffp-contract=off), because the kernels take
 * those decisions in float32 and the integer outputs must agree bit for bit.
 * The per-pixel skip/stop tests are taken in double; a pixel whose decision
 * lies within a stated relative window of its threshold is flagged
 * "ambiguous" so a float32 implementation may legitimately decide it the
 * other way.
 *
 * Readings of points the paper leaves open are listed beside each constant.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Scalar of the continuous arithmetic.  The checker is this file as it is
 * (double, single-threaded: the OpenMP pragmas below are inert without
 * -fopenmp, so every loop runs in its written order).  The CPU baseline the
 * benchmark times is the same source built with -DORC_REAL=float -fopenmp:
 * the float instantiation, parallel over Gaussians, pixel rows and map
 * entries, with per-thread gradient buffers summed in thread order.  The
 * float32 decision path is float in both. */
#ifndef ORC_REAL
#define ORC_REAL double
#endif
typedef ORC_REAL real;

static int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads the parallel loops use (1 in the checker build), and a way to set
 * them (no effect in the checker build). */
int orc_num_threads(void) { return orc_threads(); }

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static int orc_thread_id(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

/* ------------------------------------------------------------------------- */
/* Constants (the paper cites 3DGS for all of them and prints none).         */
/* ------------------------------------------------------------------------- */
#define OR_Z_NEAR_F      0.2f     /* cull depth (m)                              */
#define OR_Z_NEAR        0.2
#define OR_DILATION_F    0.3f     /* low-pass dilation of the 2-D covariance     */
#define OR_DILATION      0.3
#define OR_JCLAMP_F      1.3f     /* clamp of x/z, y/z in the EWA Jacobian       */
#define OR_JCLAMP        1.3
#define OR_EIG_FLOOR_F   0.1f     /* floor under the eigenvalue discriminant     */
#define OR_RADIUS_K_F    3.0f     /* screen radius = ceil(3 sqrt(lambda_max))    */
#define OR_ALPHA_MAX     0.99     /* alpha cap                                   */
#define OR_ALPHA_MIN     (1.0 / 255.0) /* alpha skip threshold                   */
#define OR_T_MIN         1e-4     /* transmittance stop threshold                */
#define OR_SSIM_C1       (0.01 * 0.01)
#define OR_SSIM_C2       (0.03 * 0.03)
#define OR_SSIM_WIN      11
#define OR_SSIM_SIGMA    1.5

static const double OR_PI = 3.14159265358979323846;

/* Camera: world -> camera x_c = R x_w + t (Eq. 2), pinhole pi_c.           */
typedef struct {
    double fx, fy, cx, cy;
    int32_t width, height;
    double R[9];   /* row-major */
    double t[3];
} orc_cam;

/* ------------------------------------------------------------------------- */
/* Real spherical harmonics to degree 3 (Condon-Shortley phase).             */
/* Normalisation K_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times sqrt 2  */
/* for m != 0), written as the per-polynomial factors below.                 */
/* ------------------------------------------------------------------------- */
static void sh_consts(real* k)
{
    k[0] = 0.5 * sqrt(1.0 / OR_PI);              /* Y00                  */
    k[1] = sqrt(3.0 / (4.0 * OR_PI));            /* l=1                  */
    k[2] = 0.5 * sqrt(15.0 / OR_PI);             /* xy, yz, xz           */
    k[3] = 0.25 * sqrt(5.0 / OR_PI);             /* 2z^2-x^2-y^2         */
    k[4] = 0.25 * sqrt(15.0 / OR_PI);            /* x^2-y^2              */
    k[5] = 0.25 * sqrt(35.0 / (2.0 * OR_PI));    /* y(3x^2-y^2), x(x^2-3y^2) */
    k[6] = 0.5 * sqrt(105.0 / OR_PI);            /* xyz                  */
    k[7] = 0.25 * sqrt(21.0 / (2.0 * OR_PI));    /* y(4z^2-x^2-y^2), x(...) */
    k[8] = 0.25 * sqrt(7.0 / OR_PI);             /* z(2z^2-3x^2-3y^2)    */
    k[9] = 0.25 * sqrt(105.0 / OR_PI);           /* z(x^2-y^2)           */
}

/* Y[16] at unit direction (x,y,z); dY[16][3] its gradient (may be NULL).    */
void orc_sh_basis(int deg, real x, real y, real z, real* Y, real* dY)
{
    real k[10];
    sh_consts(k);
    int nb = (deg + 1) * (deg + 1);
    real d[16][3];
    memset(d, 0, sizeof(d));
    Y[0] = k[0];
    if (deg >= 1) {
        Y[1] = -k[1] * y;  d[1][1] = -k[1];
        Y[2] =  k[1] * z;  d[2][2] =  k[1];
        Y[3] = -k[1] * x;  d[3][0] = -k[1];
    }
    if (deg >= 2) {
        Y[4] =  k[2] * x * y;                 d[4][0] = k[2] * y;  d[4][1] = k[2] * x;
        Y[5] = -k[2] * y * z;                 d[5][1] = -k[2] * z; d[5][2] = -k[2] * y;
        Y[6] =  k[3] * (2 * z * z - x * x - y * y);
        d[6][0] = -2 * k[3] * x; d[6][1] = -2 * k[3] * y; d[6][2] = 4 * k[3] * z;
        Y[7] = -k[2] * x * z;                 d[7][0] = -k[2] * z; d[7][2] = -k[2] * x;
        Y[8] =  k[4] * (x * x - y * y);       d[8][0] = 2 * k[4] * x; d[8][1] = -2 * k[4] * y;
    }
    if (deg >= 3) {
        Y[9]  = -k[5] * y * (3 * x * x - y * y);
        d[9][0] = -k[5] * 6 * x * y; d[9][1] = -k[5] * (3 * x * x - 3 * y * y);
        Y[10] =  k[6] * x * y * z;
        d[10][0] = k[6] * y * z; d[10][1] = k[6] * x * z; d[10][2] = k[6] * x * y;
        Y[11] = -k[7] * y * (4 * z * z - x * x - y * y);
        d[11][0] = -k[7] * (-2 * x * y);
        d[11][1] = -k[7] * (4 * z * z - x * x - 3 * y * y);
        d[11][2] = -k[7] * (8 * y * z);
        Y[12] =  k[8] * z * (2 * z * z - 3 * x * x - 3 * y * y);
        d[12][0] = k[8] * (-6 * x * z); d[12][1] = k[8] * (-6 * y * z);
        d[12][2] = k[8] * (6 * z * z - 3 * x * x - 3 * y * y);
        Y[13] = -k[7] * x * (4 * z * z - x * x - y * y);
        d[13][0] = -k[7] * (4 * z * z - 3 * x * x - y * y);
        d[13][1] = -k[7] * (-2 * x * y);
        d[13][2] = -k[7] * (8 * x * z);
        Y[14] =  k[9] * z * (x * x - y * y);
        d[14][0] = k[9] * 2 * x * z; d[14][1] = -k[9] * 2 * y * z; d[14][2] = k[9] * (x * x - y * y);
        Y[15] = -k[5] * x * (x * x - 3 * y * y);
        d[15][0] = -k[5] * (3 * x * x - 3 * y * y); d[15][1] = -k[5] * (-6 * x * y);
    }
    if (dY)
        for (int i = 0; i < nb; i++)
            for (int c = 0; c < 3; c++) dY[i * 3 + c] = d[i][c];
}

/* ------------------------------------------------------------------------- */
/* exp in the float32 decision path: Cody-Waite reduction x = k ln2 + r with */
/* ln2 split into a 16-bit head and a tail, then the Taylor polynomial of    */
/* exp(r) to degree 8 (coefficients 1/j!) by Horner's rule, then 2^k.  A     */
/* fixed sequence of correctly rounded float32 operations, so any IEEE       */
/* implementation of the same sequence returns the same bits; accurate to a  */
/* couple of ulp (|r| <= ln2/2, truncation r^9/9! < 1.4e-10).               */
/* ------------------------------------------------------------------------- */
float orc_expf_decision(float x)
{
    const float ln2_hi = 0.693145751953125f;      /* 45425 * 2^-16 */
    const float ln2_lo = 1.42860682030941723212e-6f;
    const float k = rintf(x * 1.44269504088896340736f);
    const float r = (x - k * ln2_hi) - k * ln2_lo;
    float p = 1.0f / 40320.0f;
    p = p * r + 1.0f / 5040.0f;
    p = p * r + 1.0f / 720.0f;
    p = p * r + 1.0f / 120.0f;
    p = p * r + 1.0f / 24.0f;
    p = p * r + 1.0f / 6.0f;
    p = p * r + 0.5f;
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    if (!(k >= -300.0f && k <= 300.0f)) return k > 0.0f ? INFINITY : 0.0f;
    return ldexpf(p, (int)k);
}

/* ------------------------------------------------------------------------- */
/* log in the float32 decision path: x = m 2^e with m in [sqrt(1/2),        */
/* sqrt(2)) taken from the bits, ln m = 2 atanh(s) with s = (m-1)/(m+1) by   */
/* its odd series to s^11 (|s| <= 0.1716, truncation 2 s^13/13 < 2e-11), then */
/* e ln2 with ln2 split as in the exp above.  A fixed sequence of correctly   */
/* rounded float32 operations.                                               */
/* ------------------------------------------------------------------------- */
float orc_logf_decision(float x)
{
    if (!(x > 0.0f)) return -INFINITY;
    if (x == INFINITY) return INFINITY;
    uint32_t bits;
    int e0 = 0;
    if (x < 1.17549435e-38f) { x = x * 16777216.0f; e0 = -24; }   /* subnormal: scale by 2^24 */
    memcpy(&bits, &x, 4);
    int e = (int)((bits >> 23) & 0xffu) - 126 + e0;
    uint32_t mb = (bits & 0x7fffffu) | 0x3f000000u;                  /* m in [0.5, 1) */
    float m;
    memcpy(&m, &mb, 4);
    if (m < 0.70710678118654752f) { m = m * 2.0f; e -= 1; }
    const float ln2_hi = 0.693145751953125f;
    const float ln2_lo = 1.42860682030941723212e-6f;
    const float sv = (m - 1.0f) / (m + 1.0f);
    const float s2 = sv * sv;
    float p = (float)(2.0 / 11.0);
    p = p * s2 + (float)(2.0 / 9.0);
    p = p * s2 + (float)(2.0 / 7.0);
    p = p * s2 + (float)(2.0 / 5.0);
    p = p * s2 + (float)(2.0 / 3.0);
    p = p * s2 + 2.0f;
    const float lm = p * sv;
    const float fe = (float)e;
    return fe * ln2_hi + (fe * ln2_lo + lm);
}

/* ------------------------------------------------------------------------- */
/* Exact tile culling, float32 decision path: can the Gaussian reach alpha   */
/* >= 1/255 at a pixel centre of the tile whose centres span [X0, X0+T1] x    */
/* [Y0, Y0+T1]?  q(d) = A dx^2 + 2B dx dy + C dy^2 (the conic) is convex, so  */
/* off the centre its minimum over the rectangle lies on an edge; on an edge  */
/* x = const the 1-D minimiser is dy = (-B/C) dx, on y = const dx = (-B/A) dy, */
/* clamped to the edge.  Kept iff that minimum is <= ks, where ks = 2 ln(255  */
/* o) with a slack of 2^-7 (relative and absolute) so that every dropped tile */
/* stays below the alpha threshold by a margin far above the rounding of the  */
/* per-pixel alpha.  cp = (u, v, A, B, C, ks, -B/C, -B/A).                    */
/* ------------------------------------------------------------------------- */
static int tile_keep(const float cp[8], float X0, float Y0, float T1)
{
    const float u = cp[0], v = cp[1], A = cp[2], B = cp[3], C = cp[4], ks = cp[5], bc = cp[6], ba = cp[7];
    const float dx0 = X0 - u, dx1 = (X0 + T1) - u, dy0 = Y0 - v, dy1 = (Y0 + T1) - v;
    if (dx0 <= 0.0f && dx1 >= 0.0f && dy0 <= 0.0f && dy1 >= 0.0f) return 1;
    const float B2 = 2.0f * B;
    float qmin = INFINITY;
    const float dxs[2] = { dx0, dx1 }, dys[2] = { dy0, dy1 };
    for (int i = 0; i < 2; i++) {
        const float dx = dxs[i];
        const float t = fminf(fmaxf(bc * dx, dy0), dy1);
        const float q = ((A * dx) * dx + (B2 * dx) * t) + (C * t) * t;
        qmin = fminf(qmin, q);
    }
    for (int i = 0; i < 2; i++) {
        const float dy = dys[i];
        const float t = fminf(fmaxf(ba * dy, dx0), dx1);
        const float q = ((A * t) * t + (B2 * t) * dy) + (C * dy) * dy;
        qmin = fminf(qmin, q);
    }
    return qmin <= ks;
}

/* ------------------------------------------------------------------------- */
/* Float32 decision path: cull, radius, rectangle, depth key (Eq. 2-3).      */
/* Returns 1 if the Gaussian is kept.                                         */
/* ------------------------------------------------------------------------- */
static int project_f32(const real* mud, const real* lsd, const real* qd, real logit,
                       const orc_cam* cam, int Ts,
                       int32_t* radius, int32_t rect[4], uint32_t* dbits, float cp[8])
{
    float R[9], t[3], mu[3], ls[3], q[4];
    for (int i = 0; i < 9; i++) R[i] = (float)cam->R[i];
    for (int i = 0; i < 3; i++) { t[i] = (float)cam->t[i]; mu[i] = (float)mud[i]; ls[i] = (float)lsd[i]; }
    for (int i = 0; i < 4; i++) q[i] = (float)qd[i];
    const float fx = (float)cam->fx, fy = (float)cam->fy, cx = (float)cam->cx, cy = (float)cam->cy;
    const int TX = (cam->width + Ts - 1) / Ts, TY = (cam->height + Ts - 1) / Ts;
    float x = ((R[0] * mu[0] + R[1] * mu[1]) + R[2] * mu[2]) + t[0];
    float y = ((R[3] * mu[0] + R[4] * mu[1]) + R[5] * mu[2]) + t[1];
    float z = ((R[6] * mu[0] + R[7] * mu[1]) + R[8] * mu[2]) + t[2];
    if (!(z > OR_Z_NEAR_F)) return 0;
    float iz = 1.0f / z;
    float xz = x * iz, yz = y * iz;
    float u = fx * xz + cx;
    float v = fy * yz + cy;
    if (!(fabsf(u) <= 3.0e38f) || !(fabsf(v) <= 3.0e38f)) return 0;

    /* Eq. 1: Sigma = R S S^T R^T, S = diag(exp(log-scale)), exp as above.   */
    float s0 = orc_expf_decision(ls[0]);
    float s1 = orc_expf_decision(ls[1]);
    float s2 = orc_expf_decision(ls[2]);
    float qq = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
    if (!(qq > 0.0f) || !(qq <= 3.0e38f)) return 0;
    float inv = 1.0f / sqrtf(qq);
    float w = q[0] * inv, qx = q[1] * inv, qy = q[2] * inv, qz = q[3] * inv;
    float r00 = 1.0f - 2.0f * (qy * qy + qz * qz);
    float r01 = 2.0f * (qx * qy - w * qz);
    float r02 = 2.0f * (qx * qz + w * qy);
    float r10 = 2.0f * (qx * qy + w * qz);
    float r11 = 1.0f - 2.0f * (qx * qx + qz * qz);
    float r12 = 2.0f * (qy * qz - w * qx);
    float r20 = 2.0f * (qx * qz - w * qy);
    float r21 = 2.0f * (qy * qz + w * qx);
    float r22 = 1.0f - 2.0f * (qx * qx + qy * qy);
    float M[9] = { r00 * s0, r01 * s1, r02 * s2,
                   r10 * s0, r11 * s1, r12 * s2,
                   r20 * s0, r21 * s1, r22 * s2 };
    float S[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            S[i * 3 + j] = (M[i * 3 + 0] * M[j * 3 + 0] + M[i * 3 + 1] * M[j * 3 + 1])
                           + M[i * 3 + 2] * M[j * 3 + 2];

    /* Eq. 3: Sigma' = [J W Sigma W^T J^T]_2x2 + dilation.                      */
    float limx = OR_JCLAMP_F * ((0.5f * (float)cam->width) / fx);
    float limy = OR_JCLAMP_F * ((0.5f * (float)cam->height) / fy);
    float cxz = fminf(fmaxf(xz, -limx), limx);
    float cyz = fminf(fmaxf(yz, -limy), limy);
    float j00 = fx * iz;
    float j02 = -(fx * cxz) * iz;
    float j11 = fy * iz;
    float j12 = -(fy * cyz) * iz;
    float T[6];
    for (int k = 0; k < 3; k++) {
        T[k]     = j00 * R[k]     + j02 * R[6 + k];
        T[3 + k] = j11 * R[3 + k] + j12 * R[6 + k];
    }
    float U[6];
    for (int i = 0; i < 2; i++)
        for (int k = 0; k < 3; k++)
            U[i * 3 + k] = (T[i * 3 + 0] * S[0 * 3 + k] + T[i * 3 + 1] * S[1 * 3 + k])
                           + T[i * 3 + 2] * S[2 * 3 + k];
    float a = ((U[0] * T[0] + U[1] * T[1]) + U[2] * T[2]) + OR_DILATION_F;
    float b = (U[0] * T[3] + U[1] * T[4]) + U[2] * T[5];
    float c = ((U[3] * T[3] + U[4] * T[4]) + U[5] * T[5]) + OR_DILATION_F;
    float det = a * c - b * b;
    if (!(det > 0.0f)) return 0;
    float mid = 0.5f * (a + c);
    float lam = mid + sqrtf(fmaxf(OR_EIG_FLOOR_F, mid * mid - det));
    float r = ceilf(OR_RADIUS_K_F * sqrtf(lam));
    if (!(r >= 1.0f) || !(r <= 3.0e38f)) return 0;

    float tsf = (float)Ts;
    float x0 = fminf(fmaxf(floorf((u - r) / tsf), 0.0f), (float)TX);
    float x1 = fminf(fmaxf(floorf(((u + r) + (tsf - 1.0f)) / tsf), 0.0f), (float)TX);
    float y0 = fminf(fmaxf(floorf((v - r) / tsf), 0.0f), (float)TY);
    float y1 = fminf(fmaxf(floorf(((v + r) + (tsf - 1.0f)) / tsf), 0.0f), (float)TY);
    rect[0] = (int32_t)x0; rect[1] = (int32_t)y0; rect[2] = (int32_t)x1; rect[3] = (int32_t)y1;
    if ((rect[2] - rect[0]) * (rect[3] - rect[1]) == 0) return 0;
    *radius = (r > 2.0e9f) ? 2000000000 : (int32_t)r;
    memcpy(dbits, &z, 4);
    /* exact tile culling inputs: mu', conic, 2 ln(255 o) with slack */
    const float og = 1.0f / (1.0f + orc_expf_decision(-(float)logit));
    const float kap = 2.0f * orc_logf_decision(255.0f * og);
    cp[0] = u;
    cp[1] = v;
    cp[2] = c / det;
    cp[3] = -b / det;
    cp[4] = a / det;
    cp[5] = kap + (kap * 0.0078125f + 0.0078125f);
    cp[6] = -cp[3] / cp[4];
    cp[7] = -cp[3] / cp[2];
    return 1;
}

/* The exact culling applies to rectangles of at most 64 tiles (a larger    */
/* one keeps all its tiles, which is always allowed: it only costs          */
/* instances).                                                               */
#define OR_CULL_MAX_TILES 64

/* Tiles of the rectangle kept by the exact culling (all with cull = 0).    */
static uint32_t kept_tiles(const int32_t rc[4], const float cp[8], int Ts, int cull)
{
    const int area = (rc[2] - rc[0]) * (rc[3] - rc[1]);
    if (!cull || area > OR_CULL_MAX_TILES) return (uint32_t)area;
    uint32_t k = 0;
    const float T1 = (float)(Ts - 1);
    for (int ty = rc[1]; ty < rc[3]; ty++)
        for (int tx = rc[0]; tx < rc[2]; tx++) k += (uint32_t)tile_keep(cp, (float)(tx * Ts), (float)(ty * Ts), T1);
    return k;
}

/* ------------------------------------------------------------------------- */
/* Double path: rotation, covariance, EWA, conic, opacity, SH colour.        */
/* ------------------------------------------------------------------------- */
static void quat_to_rot(const real* qn, real* Rm)
{
    real w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    Rm[0] = 1 - 2 * (y * y + z * z); Rm[1] = 2 * (x * y - w * z);     Rm[2] = 2 * (x * z + w * y);
    Rm[3] = 2 * (x * y + w * z);     Rm[4] = 1 - 2 * (x * x + z * z); Rm[5] = 2 * (y * z - w * x);
    Rm[6] = 2 * (x * z - w * y);     Rm[7] = 2 * (y * z + w * x);     Rm[8] = 1 - 2 * (x * x + y * y);
}

typedef struct {
    real mc[3];        /* camera-space mean mu-hat                        */
    real u, v;         /* mu'                                             */
    real s[3];         /* scales                                          */
    real qn[4];        /* unit quaternion                                 */
    real qnorm;
    real Rq[9];        /* rotation from the quaternion                    */
    real Sig[9];       /* 3-D covariance                                  */
    real J[6];         /* 2x3 EWA Jacobian (row-major), clamp applied     */
    int clx, cly;        /* 1 if the x/z (y/z) clamp is active              */
    real T[6];         /* J W                                             */
    real cov[3];       /* a, b, c of Sigma' (with dilation)               */
    real det;
    real conic[3];     /* A, B, C                                         */
    real o;            /* opacity                                         */
    real dir[3];       /* unit view direction                             */
    real dnorm;
    real rgb[3];
    int clamp[3];        /* 1 where rgb was clamped at 0                    */
    real Y[16];
} geom_t;

static void project_f64(const real* mu, const real* ls, const real* q, real logit,
                        const real* sh, int deg, const orc_cam* cam, geom_t* G)
{
    real R[9], t[3];
    for (int i = 0; i < 9; i++) R[i] = cam->R[i];
    for (int i = 0; i < 3; i++) t[i] = cam->t[i];
    real m[3] = { mu[0], mu[1], mu[2] };
    for (int i = 0; i < 3; i++)
        G->mc[i] = R[i * 3 + 0] * m[0] + R[i * 3 + 1] * m[1] + R[i * 3 + 2] * m[2] + t[i];
    real x = G->mc[0], y = G->mc[1], z = G->mc[2];
    real fx = cam->fx, fy = cam->fy;
    G->u = fx * x / z + cam->cx;
    G->v = fy * y / z + cam->cy;
    for (int i = 0; i < 3; i++) G->s[i] = exp(ls[i]);
    real qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    G->qnorm = sqrt(qq);
    for (int i = 0; i < 4; i++) G->qn[i] = q[i] / G->qnorm;
    quat_to_rot(G->qn, G->Rq);
    real M[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) M[i * 3 + j] = G->Rq[i * 3 + j] * G->s[j];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            G->Sig[i * 3 + j] = M[i * 3 + 0] * M[j * 3 + 0] + M[i * 3 + 1] * M[j * 3 + 1]
                                + M[i * 3 + 2] * M[j * 3 + 2];
    real limx = OR_JCLAMP * (0.5 * cam->width / fx);
    real limy = OR_JCLAMP * (0.5 * cam->height / fy);
    real xz = x / z, yz = y / z;
    G->clx = (xz < -limx || xz > limx);
    G->cly = (yz < -limy || yz > limy);
    real cxz = xz < -limx ? -limx : (xz > limx ? limx : xz);
    real cyz = yz < -limy ? -limy : (yz > limy ? limy : yz);
    G->J[0] = fx / z; G->J[1] = 0; G->J[2] = -fx * cxz / z;
    G->J[3] = 0; G->J[4] = fy / z; G->J[5] = -fy * cyz / z;
    for (int i = 0; i < 2; i++)
        for (int k = 0; k < 3; k++)
            G->T[i * 3 + k] = G->J[i * 3 + 0] * R[k] + G->J[i * 3 + 1] * R[3 + k]
                              + G->J[i * 3 + 2] * R[6 + k];
    real U[6];
    for (int i = 0; i < 2; i++)
        for (int k = 0; k < 3; k++)
            U[i * 3 + k] = G->T[i * 3 + 0] * G->Sig[k] + G->T[i * 3 + 1] * G->Sig[3 + k]
                           + G->T[i * 3 + 2] * G->Sig[6 + k];
    G->cov[0] = U[0] * G->T[0] + U[1] * G->T[1] + U[2] * G->T[2] + OR_DILATION;
    G->cov[1] = U[0] * G->T[3] + U[1] * G->T[4] + U[2] * G->T[5];
    G->cov[2] = U[3] * G->T[3] + U[4] * G->T[4] + U[5] * G->T[5] + OR_DILATION;
    G->det = G->cov[0] * G->cov[2] - G->cov[1] * G->cov[1];
    G->conic[0] = G->cov[2] / G->det;
    G->conic[1] = -G->cov[1] / G->det;
    G->conic[2] = G->cov[0] / G->det;
    G->o = 1.0 / (1.0 + exp(-logit));

    /* SH colour: direction from the camera centre c_w = -R^T t to the mean.  */
    real cw[3];
    for (int i = 0; i < 3; i++) cw[i] = -(R[0 * 3 + i] * t[0] + R[1 * 3 + i] * t[1] + R[2 * 3 + i] * t[2]);
    real d[3] = { m[0] - cw[0], m[1] - cw[1], m[2] - cw[2] };
    G->dnorm = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int i = 0; i < 3; i++) G->dir[i] = d[i] / G->dnorm;
    orc_sh_basis(deg, G->dir[0], G->dir[1], G->dir[2], G->Y, NULL);
    int nb = (deg + 1) * (deg + 1);
    for (int c = 0; c < 3; c++) {
        real acc = 0.5;
        for (int k = 0; k < nb; k++) acc += G->Y[k] * sh[k * 3 + c];
        G->clamp[c] = acc < 0.0;
        G->rgb[c] = acc < 0.0 ? 0.0 : acc;
    }
}

/* ------------------------------------------------------------------------- */
/* Preprocess every Gaussian.                                                */
/* ------------------------------------------------------------------------- */
/* cull = 1: exact tile culling (touched counts only the kept tiles; cullp, */
/* 8 floats per Gaussian, holds the test's inputs for orc_bin).              */
void orc_preprocess(int64_t n, int deg, const real* means, const real* lscale,
                    const real* quat, const real* logit, const real* sh,
                    const orc_cam* cam, int Ts, int cull,
                    int32_t* radius, int32_t* rect, uint32_t* touched, uint32_t* dbits,
                    real* mean2d, real* conic, real* opac, real* rgb, real* depth,
                    uint8_t* flags, float* cullp)
{
    int nb = (deg + 1) * (deg + 1);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; g++) {
        int32_t r = 0, rc[4] = { 0, 0, 0, 0 };
        uint32_t db = 0;
        float cp[8] = { 0, 0, 0, 0, 0, 0, 0, 0 };
        int keep = project_f32(means + 3 * g, lscale + 3 * g, quat + 4 * g, logit[g], cam, Ts, &r, rc, &db, cp);
        radius[g] = keep ? r : 0;
        for (int i = 0; i < 4; i++) rect[4 * g + i] = keep ? rc[i] : 0;
        touched[g] = keep ? kept_tiles(rc, cp, Ts, cull) : 0;
        for (int i = 0; i < 8; i++) cullp[8 * g + i] = keep ? cp[i] : 0.0f;
        dbits[g] = keep ? db : 0;
        if (keep) {
            geom_t G;
            project_f64(means + 3 * g, lscale + 3 * g, quat + 4 * g, logit[g], sh + (size_t)nb * 3 * g,
                        deg, cam, &G);
            mean2d[2 * g] = G.u; mean2d[2 * g + 1] = G.v;
            for (int i = 0; i < 3; i++) { conic[3 * g + i] = G.conic[i]; rgb[3 * g + i] = G.rgb[i]; }
            opac[g] = G.o;
            depth[g] = G.mc[2];
            if (flags)
                flags[g] = (uint8_t)(G.clamp[0] | (G.clamp[1] << 1) | (G.clamp[2] << 2)
                                     | (G.clx << 3) | (G.cly << 4));
        } else {
            mean2d[2 * g] = mean2d[2 * g + 1] = 0;
            for (int i = 0; i < 3; i++) { conic[3 * g + i] = 0; rgb[3 * g + i] = 0; }
            opac[g] = 0; depth[g] = 0;
            if (flags) flags[g] = 0;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Binning: duplicate (tile | depth) keys, stable sort, per-tile ranges.     */
/* ------------------------------------------------------------------------- */
typedef struct { uint64_t key; uint64_t order; uint32_t val; } inst_t;

static int inst_cmp(const void* a, const void* b)
{
    const inst_t* x = (const inst_t*)a;
    const inst_t* y = (const inst_t*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->order != y->order) return x->order < y->order ? -1 : 1;
    return 0;
}

int64_t orc_num_instances(int64_t n, const uint32_t* touched)
{
    int64_t s = 0;
    for (int64_t g = 0; g < n; g++) s += touched[g];
    return s;
}

/* keys/vals sized orc_num_instances(); ranges sized 2 * num_tiles.  With   */
/* cullp (from orc_preprocess with cull = 1) only the kept tiles are emitted. */
/* Only tiles t with t % tile_step == 0 get instances (1: all of them; a     */
/* larger step is the benchmark's sample of the work); returns the number   */
/* emitted.                                                                  */
int64_t orc_bin(int64_t n, const int32_t* rect, const uint32_t* touched, const uint32_t* dbits,
                const float* cullp, int Ts, int TX, int TY, int tile_step, uint64_t* keys, uint32_t* vals,
                uint32_t* ranges)
{
    int64_t ninst = orc_num_instances(n, touched);
    inst_t* buf = (inst_t*)malloc(sizeof(inst_t) * (size_t)(ninst > 0 ? ninst : 1));
    int64_t k = 0;
    for (int64_t g = 0; g < n; g++) {
        if (!touched[g]) continue;
        const int32_t* rc = rect + 4 * g;
        const int culled = cullp && (rc[2] - rc[0]) * (rc[3] - rc[1]) <= OR_CULL_MAX_TILES;
        for (int ty = rc[1]; ty < rc[3]; ty++)
            for (int tx = rc[0]; tx < rc[2]; tx++) {
                if (culled && !tile_keep(cullp + 8 * g, (float)(tx * Ts), (float)(ty * Ts), (float)(Ts - 1)))
                    continue;
                if ((ty * TX + tx) % tile_step) continue;
                buf[k].key = ((uint64_t)(uint32_t)(ty * TX + tx) << 32) | (uint64_t)dbits[g];
                buf[k].order = (uint64_t)k;
                buf[k].val = (uint32_t)g;
                k++;
            }
    }
    ninst = k;
    qsort(buf, (size_t)ninst, sizeof(inst_t), inst_cmp);
    int nt = TX * TY;
    for (int i = 0; i < 2 * nt; i++) ranges[i] = 0;
    for (int64_t i = 0; i < ninst; i++) {
        keys[i] = buf[i].key;
        vals[i] = buf[i].val;
        uint32_t tile = (uint32_t)(buf[i].key >> 32);
        if (i == 0 || (uint32_t)(buf[i - 1].key >> 32) != tile) ranges[2 * tile] = (uint32_t)i;
        if (i == ninst - 1 || (uint32_t)(buf[i + 1].key >> 32) != tile) ranges[2 * tile + 1] = (uint32_t)(i + 1);
    }
    free(buf);
    return ninst;
}

/* ------------------------------------------------------------------------- */
/* Compositing (Eq. 4-7), one pixel.  Records the contributors for reuse by  */
/* the backward.  Returns the number of contributors written to `list`.      */
/* ------------------------------------------------------------------------- */
typedef struct {
    real amb_alpha_rel;   /* relative window around the alpha threshold  */
    real amb_T_rel;       /* relative window around the T threshold      */
} orc_amb;

static int composite_pixel(real px, real py, const uint32_t* idx, int64_t cnt,
                           const real* mean2d, const real* conic, const real* opac,
                           const real* rgb, const real* depth,
                           real* C, real* D, real* O, real* Tfin, int32_t* ncontrib,
                           uint8_t* amb, const orc_amb* ab,
                           int64_t* list_pos, real* list_alpha, real* list_T, int* list_capped,
                           real* list_G, uint64_t* sig)
{
    real T = 1.0, c0 = 0, c1 = 0, c2 = 0, dd = 0, oo = 0;
    int32_t last = 0;
    int nl = 0;
    uint8_t a = 0;
    uint64_t h = 1469598103934665603ULL;   /* FNV-1a over (position, capped) */
    for (int64_t i = 0; i < cnt; i++) {
        uint32_t g = idx[i];
        real dx = mean2d[2 * g] - px, dy = mean2d[2 * g + 1] - py;
        real A = conic[3 * g], B = conic[3 * g + 1], Cc = conic[3 * g + 2];
        real power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
        real scale = 0.5 * (fabs(A * dx * dx) + fabs(Cc * dy * dy)) + fabs(B * dx * dy);
        if (fabs(power) <= 1e-6 * scale + 1e-30 && power <= 0.0 && scale > 0) a = 1;
        if (power > 0.0) { if (power <= 1e-6 * scale) a = 1; continue; }
        real G = exp(power);
        real araw = opac[g] * G;
        if (fabs(araw - OR_ALPHA_MIN) <= ab->amb_alpha_rel * OR_ALPHA_MIN) a = 1;
        real alpha = araw < OR_ALPHA_MAX ? araw : OR_ALPHA_MAX;
        if (alpha < OR_ALPHA_MIN) continue;
        real test_T = T * (1.0 - alpha);
        if (fabs(test_T - OR_T_MIN) <= ab->amb_T_rel * OR_T_MIN) a = 1;
        if (test_T < OR_T_MIN) break;
        real w = alpha * T;
        c0 += rgb[3 * g] * w; c1 += rgb[3 * g + 1] * w; c2 += rgb[3 * g + 2] * w;
        dd += depth[g] * w; oo += w;
        if (list_pos) {
            list_pos[nl] = i; list_alpha[nl] = alpha; list_T[nl] = T;
            list_capped[nl] = araw >= OR_ALPHA_MAX; list_G[nl] = G;
        }
        h = (h ^ (uint64_t)(2 * i + (araw >= OR_ALPHA_MAX))) * 1099511628211ULL;
        nl++;
        T = test_T;
        last = (int32_t)(i + 1);
    }
    C[0] = c0; C[1] = c1; C[2] = c2;
    *D = dd; *O = oo; *Tfin = T; *ncontrib = last;
    *amb = a;
    if (sig) *sig = h;
    return nl;
}

/* Pixels of tiles t with t % tile_step != 0 are left untouched.           */
void orc_render(int W, int H, int Ts, int tile_step, const uint32_t* vals, const uint32_t* ranges,
                const real* mean2d, const real* conic, const real* opac,
                const real* rgb, const real* depth,
                real amb_alpha_rel, real amb_T_rel,
                real* C, real* D, real* O, real* Tfin, int32_t* ncontrib, uint8_t* amb,
                uint64_t* sig)
{
    int TX = (W + Ts - 1) / Ts;
    orc_amb ab = { amb_alpha_rel, amb_T_rel };
#pragma omp parallel for schedule(dynamic, 1)
    for (int py = 0; py < H; py++)
        for (int px = 0; px < W; px++) {
            int tile = (py / Ts) * TX + (px / Ts);
            if (tile % tile_step) continue;
            uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
            size_t p = (size_t)py * W + px;
            composite_pixel((real)px, (real)py, vals + s, (int64_t)e - s, mean2d, conic, opac,
                            rgb, depth, C + 3 * p, D + p, O + p, Tfin + p, ncontrib + p, amb + p, &ab,
                            NULL, NULL, NULL, NULL, NULL, sig ? sig + p : NULL);
        }
}

/* Brute force (pin only): per pixel, every Gaussian whose rectangle holds   */
/* the pixel's tile, ordered by (depth bits, index), composited directly.     */
typedef struct { uint32_t db; uint32_t g; } dg_t;
static int dg_cmp(const void* a, const void* b)
{
    const dg_t* x = (const dg_t*)a;
    const dg_t* y = (const dg_t*)b;
    if (x->db != y->db) return x->db < y->db ? -1 : 1;
    return x->g < y->g ? -1 : (x->g > y->g);
}

void orc_render_bruteforce(int W, int H, int Ts, int64_t n, const int32_t* rect,
                           const uint32_t* touched, const uint32_t* dbits,
                           const real* mean2d, const real* conic, const real* opac,
                           const real* rgb, const real* depth, int use_rect,
                           real* C, real* D, real* O, real* Tfin, int32_t* ncontrib)
{
    dg_t* lst = (dg_t*)malloc(sizeof(dg_t) * (size_t)(n > 0 ? n : 1));
    uint32_t* ids = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    orc_amb ab = { 0, 0 };
    for (int py = 0; py < H; py++)
        for (int px = 0; px < W; px++) {
            int tx = px / Ts, ty = py / Ts;
            int64_t m = 0;
            for (int64_t g = 0; g < n; g++) {
                if (!touched[g]) continue;
                const int32_t* rc = rect + 4 * g;
                if (use_rect && !(tx >= rc[0] && tx < rc[2] && ty >= rc[1] && ty < rc[3])) continue;
                lst[m].db = dbits[g]; lst[m].g = (uint32_t)g; m++;
            }
            qsort(lst, (size_t)m, sizeof(dg_t), dg_cmp);
            for (int64_t i = 0; i < m; i++) ids[i] = lst[i].g;
            size_t p = (size_t)py * W + px;
            uint8_t a;
            composite_pixel((real)px, (real)py, ids, m, mean2d, conic, opac, rgb, depth,
                            C + 3 * p, D + p, O + p, Tfin + p, ncontrib + p, &a, &ab,
                            NULL, NULL, NULL, NULL, NULL, NULL);
        }
    free(lst);
    free(ids);
}

/* ------------------------------------------------------------------------- */
/* Exposure + L1 + D-SSIM loss (Eq. 9) and its exact adjoint.                */
/* E is 3x4 row-major [A | b]; C_hat = A C + b.                               */
/* ------------------------------------------------------------------------- */
static void ssim_window(real* w)
{
    real s = 0;
    for (int i = 0; i < OR_SSIM_WIN; i++) {
        real d = i - OR_SSIM_WIN / 2;
        w[i] = exp(-d * d / (2.0 * OR_SSIM_SIGMA * OR_SSIM_SIGMA));
        s += w[i];
    }
    for (int i = 0; i < OR_SSIM_WIN; i++) w[i] /= s;
}

/* Zero-padded "same" 2-D correlation with the separable window (one map). */
static void blur(int W, int H, const real* in, real* out, const real* w, real* tmp)
{
    int h = OR_SSIM_WIN / 2;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            real s = 0;
            for (int k = -h; k <= h; k++) {
                int xx = x + k;
                if (xx >= 0 && xx < W) s += w[k + h] * in[(size_t)y * W + xx];
            }
            tmp[(size_t)y * W + x] = s;
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            real s = 0;
            for (int k = -h; k <= h; k++) {
                int yy = y + k;
                if (yy >= 0 && yy < H) s += w[k + h] * tmp[(size_t)yy * W + x];
            }
            out[(size_t)y * W + x] = s;
        }
}

real orc_loss(int W, int H, const real* C, const float* target, const float* E, real lambda,
                real* dL_dC, real* dL_dE, real* ssim_mean_out, real* l1_out)
{
    size_t P = (size_t)W * H;
    real w[OR_SSIM_WIN];
    ssim_window(w);
    real* Ch = (real*)malloc(sizeof(real) * P * 3);
    real* gCh = (real*)calloc(P * 3, sizeof(real));
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < P; p++)
        for (int i = 0; i < 3; i++)
            Ch[3 * p + i] = E[4 * i + 0] * C[3 * p + 0] + E[4 * i + 1] * C[3 * p + 1]
                            + E[4 * i + 2] * C[3 * p + 2] + E[4 * i + 3];
    real l1 = 0;
    real inv = 1.0 / (3.0 * (real)P);
#pragma omp parallel for schedule(static) reduction(+ : l1)
    for (size_t p = 0; p < 3 * P; p++) {
        real d = Ch[p] - (real)target[p];
        l1 += fabs(d);
        gCh[p] += (1.0 - lambda) * inv * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0));
    }
    l1 *= inv;

    real *x = malloc(sizeof(real) * P), *y = malloc(sizeof(real) * P), *tmp = malloc(sizeof(real) * P);
    real *mx = malloc(sizeof(real) * P), *my = malloc(sizeof(real) * P);
    real *exx = malloc(sizeof(real) * P), *eyy = malloc(sizeof(real) * P), *exy = malloc(sizeof(real) * P);
    real *buf = malloc(sizeof(real) * P);
    real *ga = malloc(sizeof(real) * P), *gb = malloc(sizeof(real) * P), *gc = malloc(sizeof(real) * P);
    real *ba = malloc(sizeof(real) * P), *bb = malloc(sizeof(real) * P), *bc = malloc(sizeof(real) * P);
    real ssim_sum = 0;
    real gS = -lambda * inv;     /* dL / dS(p, channel) */
    for (int ch = 0; ch < 3; ch++) {
#pragma omp parallel for schedule(static)
        for (size_t p = 0; p < P; p++) { x[p] = Ch[3 * p + ch]; y[p] = target[3 * p + ch]; }
        blur(W, H, x, mx, w, tmp);
        blur(W, H, y, my, w, tmp);
#pragma omp parallel for schedule(static)
        for (size_t p = 0; p < P; p++) buf[p] = x[p] * x[p];
        blur(W, H, buf, exx, w, tmp);
#pragma omp parallel for schedule(static)
        for (size_t p = 0; p < P; p++) buf[p] = y[p] * y[p];
        blur(W, H, buf, eyy, w, tmp);
#pragma omp parallel for schedule(static)
        for (size_t p = 0; p < P; p++) buf[p] = x[p] * y[p];
        blur(W, H, buf, exy, w, tmp);
#pragma omp parallel for schedule(static) reduction(+ : ssim_sum)
        for (size_t p = 0; p < P; p++) {
            real sxx = exx[p] - mx[p] * mx[p];
            real syy = eyy[p] - my[p] * my[p];
            real sxy = exy[p] - mx[p] * my[p];
            real N1 = 2 * mx[p] * my[p] + OR_SSIM_C1, N2 = 2 * sxy + OR_SSIM_C2;
            real D1 = mx[p] * mx[p] + my[p] * my[p] + OR_SSIM_C1, D2 = sxx + syy + OR_SSIM_C2;
            real S = N1 * N2 / (D1 * D2);
            ssim_sum += S;
            /* partials w.r.t. mu_x, E[x^2], E[xy] (mu_y, E[y^2] are constants) */
            real dS_dN1 = N2 / (D1 * D2), dS_dN2 = N1 / (D1 * D2);
            real dS_dD1 = -S / D1, dS_dD2 = -S / D2;
            real dmx = dS_dN1 * 2 * my[p] + dS_dN2 * (-2 * my[p]) + dS_dD1 * 2 * mx[p]
                         + dS_dD2 * (-2 * mx[p]);
            real dexx = dS_dD2;
            real dexy = dS_dN2 * 2;
            ga[p] = gS * dmx; gb[p] = gS * dexx; gc[p] = gS * dexy;
        }
        blur(W, H, ga, ba, w, tmp);
        blur(W, H, gb, bb, w, tmp);
        blur(W, H, gc, bc, w, tmp);
#pragma omp parallel for schedule(static)
        for (size_t p = 0; p < P; p++) gCh[3 * p + ch] += ba[p] + 2 * x[p] * bb[p] + y[p] * bc[p];
    }
    real ssim_mean = ssim_sum * inv;
    real loss = (1.0 - lambda) * l1 + lambda * (1.0 - ssim_mean);

    for (int i = 0; i < 12; i++) dL_dE[i] = 0;
#pragma omp parallel for schedule(static) reduction(+ : dL_dE[:12])
    for (size_t p = 0; p < P; p++)
        for (int i = 0; i < 3; i++) {
            real g = gCh[3 * p + i];
            dL_dE[4 * i + 0] += g * C[3 * p + 0];
            dL_dE[4 * i + 1] += g * C[3 * p + 1];
            dL_dE[4 * i + 2] += g * C[3 * p + 2];
            dL_dE[4 * i + 3] += g;
        }
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < P; p++)
        for (int j = 0; j < 3; j++)
            dL_dC[3 * p + j] = E[0 * 4 + j] * gCh[3 * p + 0] + E[1 * 4 + j] * gCh[3 * p + 1]
                               + E[2 * 4 + j] * gCh[3 * p + 2];
    if (ssim_mean_out) *ssim_mean_out = ssim_mean;
    if (l1_out) *l1_out = l1;
    free(Ch); free(gCh); free(x); free(y); free(tmp); free(mx); free(my); free(exx); free(eyy);
    free(exy); free(buf); free(ga); free(gb); free(gc); free(ba); free(bb); free(bc);
    return loss;
}

/* ------------------------------------------------------------------------- */
/* Backward.  Per pixel, the contributor list is replayed in real; each    */
/* contributor receives dL/d(mu'), dL/d(conic), dL/d(o), dL/d(rgb),          */
/* dL/d(depth); the chain rule then reaches the parameters and the pose.     */
/* g2d layout per Gaussian: [du, dv, dA, dB, dC, do, dr, dg, db, dz].         */
/* ------------------------------------------------------------------------- */
/* Pixels of tiles t with t % tile_step != 0 contribute nothing.  Built   */
/* with OpenMP, each thread sums into its own buffer and the buffers are    */
/* added in thread order; the checker build sums in pixel order directly.   */
void orc_backward_2d(int W, int H, int Ts, int tile_step, const uint32_t* vals, const uint32_t* ranges,
                     const real* mean2d, const real* conic, const real* opac,
                     const real* rgb, const real* depth,
                     const real* dL_dC, const real* dL_dD, const real* dL_dO,
                     int64_t n, real* g2d)
{
    int TX = (W + Ts - 1) / Ts;
    memset(g2d, 0, sizeof(real) * 10 * (size_t)n);
    int64_t maxc = 0;
    int nt = TX * ((H + Ts - 1) / Ts);
    for (int t = 0; t < nt; t++) {
        int64_t c = (int64_t)ranges[2 * t + 1] - ranges[2 * t];
        if (c > maxc) maxc = c;
    }
    const int nth = orc_threads();
    real* acc = nth > 1 ? (real*)calloc((size_t)nth * 10 * (size_t)n, sizeof(real)) : g2d;
#pragma omp parallel num_threads(nth)
    {
        real* gg = nth > 1 ? acc + (size_t)orc_thread_id() * 10 * (size_t)n : g2d;
        int64_t* lp = malloc(sizeof(int64_t) * (size_t)(maxc + 1));
        real* la = malloc(sizeof(real) * (size_t)(maxc + 1));
        real* lT = malloc(sizeof(real) * (size_t)(maxc + 1));
        real* lG = malloc(sizeof(real) * (size_t)(maxc + 1));
        int* lc = malloc(sizeof(int) * (size_t)(maxc + 1));
        orc_amb ab = { 0, 0 };
#pragma omp for schedule(dynamic, 1)
        for (int py = 0; py < H; py++)
            for (int px = 0; px < W; px++) {
                int tile = (py / Ts) * TX + (px / Ts);
                if (tile % tile_step) continue;
                uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
                size_t p = (size_t)py * W + px;
                real Cp[3], Dp, Op, Tf; int32_t nc; uint8_t a;
                int nl = composite_pixel((real)px, (real)py, vals + s, (int64_t)e - s, mean2d, conic,
                                         opac, rgb, depth, Cp, &Dp, &Op, &Tf, &nc, &a, &ab,
                                         lp, la, lT, lc, lG, NULL);
                real gC[3] = { dL_dC[3 * p], dL_dC[3 * p + 1], dL_dC[3 * p + 2] };
                real gD = dL_dD ? dL_dD[p] : 0.0, gO = dL_dO ? dL_dO[p] : 0.0;
                /* suffix sums: S_after = sum_{j>i} x_j alpha_j T_j (background 0) */
                real sc[3] = { 0, 0, 0 }, sd = 0, so = 0;
                for (int k = nl - 1; k >= 0; k--) {
                    uint32_t g = vals[s + lp[k]];
                    real al = la[k], T = lT[k], w = al * T;
                    real dalpha = 0;
                    for (int c = 0; c < 3; c++) {
                        dalpha += gC[c] * (T * rgb[3 * g + c] - sc[c] / (1.0 - al));
                        gg[10 * g + 6 + c] += w * gC[c];
                    }
                    dalpha += gD * (T * depth[g] - sd / (1.0 - al));
                    dalpha += gO * (T - so / (1.0 - al));
                    gg[10 * g + 9] += w * gD;
                    for (int c = 0; c < 3; c++) sc[c] += rgb[3 * g + c] * w;
                    sd += depth[g] * w; so += w;
                    if (lc[k]) continue;      /* cap active: alpha is constant */
                    real dx = mean2d[2 * g] - px, dy = mean2d[2 * g + 1] - py;
                    real A = conic[3 * g], B = conic[3 * g + 1], Cc = conic[3 * g + 2];
                    real dpow = dalpha * al;       /* d alpha / d power = alpha */
                    gg[10 * g + 5] += dalpha * lG[k];
                    gg[10 * g + 0] += dpow * (-A * dx - B * dy);
                    gg[10 * g + 1] += dpow * (-Cc * dy - B * dx);
                    gg[10 * g + 2] += dpow * (-0.5 * dx * dx);
                    gg[10 * g + 3] += dpow * (-dx * dy);
                    gg[10 * g + 4] += dpow * (-0.5 * dy * dy);
                }
            }
        free(lp); free(la); free(lT); free(lG); free(lc);
    }
    if (nth > 1) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < 10 * n; i++) {
            real t = 0;
            for (int th = 0; th < nth; th++) t += acc[(size_t)th * 10 * (size_t)n + (size_t)i];
            g2d[i] = t;
        }
        free(acc);
    }
}

/* From the 2-D gradients to the parameters (Eq. 1-3, SH) and the pose.      */
/* Pose: left perturbation T_cw <- exp(xi^) T_cw, xi = (rho, phi), at xi = 0. */
void orc_backward_params(int64_t n, int deg, const real* means, const real* lscale,
                         const real* quat, const real* logit, const real* sh,
                         const orc_cam* cam, const int32_t* radius, const real* g2d,
                         real* g_means, real* g_lscale, real* g_quat, real* g_logit,
                         real* g_sh, real* g_pose)
{
    int nb = (deg + 1) * (deg + 1);
    real R[9];
    for (int i = 0; i < 9; i++) R[i] = cam->R[i];
    for (int i = 0; i < 6; i++) g_pose[i] = 0;
    const int nth = orc_threads();
    real* pose_part = (real*)calloc((size_t)nth * 6, sizeof(real));
#pragma omp parallel num_threads(nth)
    {
    real* gp = pose_part + 6 * orc_thread_id();
#pragma omp for schedule(static)
    for (int64_t g = 0; g < n; g++) {
        real* gm = g_means + 3 * g;
        real* gl = g_lscale + 3 * g;
        real* gq = g_quat + 4 * g;
        real* gs = g_sh + (size_t)nb * 3 * g;
        for (int i = 0; i < 3; i++) { gm[i] = 0; gl[i] = 0; }
        for (int i = 0; i < 4; i++) gq[i] = 0;
        for (int i = 0; i < nb * 3; i++) gs[i] = 0;
        g_logit[g] = 0;
        if (radius[g] <= 0) continue;
        geom_t G;
        project_f64(means + 3 * g, lscale + 3 * g, quat + 4 * g, logit[g], sh + (size_t)nb * 3 * g,
                    deg, cam, &G);
        const real* d2 = g2d + 10 * g;
        real x = G.mc[0], y = G.mc[1], z = G.mc[2];
        real fx = cam->fx, fy = cam->fy;

        /* opacity */
        g_logit[g] = d2[5] * G.o * (1.0 - G.o);

        /* colour -> SH and view direction */
        real grgb[3];
        for (int c = 0; c < 3; c++) grgb[c] = G.clamp[c] ? 0.0 : d2[6 + c];
        real dY[48], Y[16];
        orc_sh_basis(deg, G.dir[0], G.dir[1], G.dir[2], Y, dY);
        real gdir[3] = { 0, 0, 0 };
        for (int k = 0; k < nb; k++)
            for (int c = 0; c < 3; c++) {
                gs[k * 3 + c] = Y[k] * grgb[c];
                real coef = sh[(size_t)nb * 3 * g + k * 3 + c] * grgb[c];
                for (int j = 0; j < 3; j++) gdir[j] += coef * dY[k * 3 + j];
            }
        /* d = dir_unnormalised / |.|: dL/d(unnormalised) = (I - d d^T) gdir / |.| */
        real dd = G.dir[0] * gdir[0] + G.dir[1] * gdir[1] + G.dir[2] * gdir[2];
        real gdu[3];
        for (int j = 0; j < 3; j++) gdu[j] = (gdir[j] - G.dir[j] * dd) / G.dnorm;
        /* dir_unnormalised = mu - c_w; c_w moves by -R^T rho under the pose twist */
        for (int j = 0; j < 3; j++) gm[j] += gdu[j];
        for (int i = 0; i < 3; i++)
            gp[i] += R[i * 3 + 0] * gdu[0] + R[i * 3 + 1] * gdu[1] + R[i * 3 + 2] * gdu[2];

        /* conic (A,B,C) -> Sigma' (a,b,c) */
        real a = G.cov[0], b = G.cov[1], c = G.cov[2], det = G.det, d2i = 1.0 / (det * det);
        real gA = d2[2], gB = d2[3], gC = d2[4];
        real ga = gA * (-c * c * d2i) + gB * (b * c * d2i) + gC * (-b * b * d2i);
        real gb = gA * (2 * b * c * d2i) + gB * (-(a * c + b * b) * d2i) + gC * (2 * a * b * d2i);
        real gc = gA * (-b * b * d2i) + gB * (a * b * d2i) + gC * (-a * a * d2i);
        /* symmetric gradient matrix of the 2x2 Sigma' */
        real Gm[4] = { ga, 0.5 * gb, 0.5 * gb, gc };
        /* Sigma' = T Sigma T^T: dL/dSigma = T^T G T; dL/dT = 2 G T Sigma      */
        real gSig[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                real s = 0;
                for (int p = 0; p < 2; p++)
                    for (int q = 0; q < 2; q++) s += G.T[p * 3 + i] * Gm[p * 2 + q] * G.T[q * 3 + j];
                gSig[i * 3 + j] = s;
            }
        real TS[6];
        for (int p = 0; p < 2; p++)
            for (int j = 0; j < 3; j++) {
                real s = 0;
                for (int k = 0; k < 3; k++) s += G.T[p * 3 + k] * G.Sig[k * 3 + j];
                TS[p * 3 + j] = s;
            }
        real gT[6];
        for (int p = 0; p < 2; p++)
            for (int j = 0; j < 3; j++)
                gT[p * 3 + j] = 2.0 * (Gm[p * 2 + 0] * TS[0 * 3 + j] + Gm[p * 2 + 1] * TS[1 * 3 + j]);
        /* Sigma = M M^T, M = Rq diag(s): dL/dM = 2 gSig M                      */
        real M[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) M[i * 3 + j] = G.Rq[i * 3 + j] * G.s[j];
        real gM[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                real s = 0;
                for (int k = 0; k < 3; k++) s += gSig[i * 3 + k] * M[k * 3 + j];
                gM[i * 3 + j] = 2.0 * s;
            }
        real gRq[9];
        for (int j = 0; j < 3; j++) {
            real s = 0;
            for (int i = 0; i < 3; i++) {
                s += gM[i * 3 + j] * G.Rq[i * 3 + j];
                gRq[i * 3 + j] = gM[i * 3 + j] * G.s[j];
            }
            gl[j] = s * G.s[j];    /* s = exp(log-scale) */
        }
        /* rotation matrix -> unit quaternion -> raw quaternion */
        real w = G.qn[0], qx = G.qn[1], qy = G.qn[2], qz = G.qn[3];
        real gn[4];
        gn[0] = 2 * (-qz * gRq[1] + qy * gRq[2] + qz * gRq[3] - qx * gRq[5] - qy * gRq[6] + qx * gRq[7]);
        gn[1] = 2 * (qy * gRq[1] + qz * gRq[2] + qy * gRq[3] - 2 * qx * gRq[4] - w * gRq[5]
                     + qz * gRq[6] + w * gRq[7] - 2 * qx * gRq[8]);
        gn[2] = 2 * (-2 * qy * gRq[0] + qx * gRq[1] + w * gRq[2] + qx * gRq[3] + qz * gRq[5]
                     - w * gRq[6] + qz * gRq[7] - 2 * qy * gRq[8]);
        gn[3] = 2 * (-2 * qz * gRq[0] - w * gRq[1] + qx * gRq[2] + w * gRq[3] - 2 * qz * gRq[4]
                     + qy * gRq[5] + qx * gRq[6] + qy * gRq[7]);
        real qdot = G.qn[0] * gn[0] + G.qn[1] * gn[1] + G.qn[2] * gn[2] + G.qn[3] * gn[3];
        for (int i = 0; i < 4; i++) gq[i] = (gn[i] - G.qn[i] * qdot) / G.qnorm;

        /* T = J W: dL/dJ = gT W^T (only the 4 non-zero entries), dL/dW = J^T gT */
        real gJ00 = 0, gJ02 = 0, gJ11 = 0, gJ12 = 0;
        for (int k = 0; k < 3; k++) {
            gJ00 += gT[k] * R[k];
            gJ02 += gT[k] * R[6 + k];
            gJ11 += gT[3 + k] * R[3 + k];
            gJ12 += gT[3 + k] * R[6 + k];
        }
        real gW[9];
        for (int r = 0; r < 3; r++)
            for (int k = 0; k < 3; k++)
                gW[r * 3 + k] = G.J[0 * 3 + r] * gT[0 * 3 + k] + G.J[1 * 3 + r] * gT[1 * 3 + k];

        /* camera-space mean: through mu', J and the depth output */
        real gmc[3] = { 0, 0, 0 };
        gmc[0] += d2[0] * fx / z;
        gmc[1] += d2[1] * fy / z;
        gmc[2] += -d2[0] * fx * x / (z * z) - d2[1] * fy * y / (z * z);
        gmc[2] += d2[9];
        gmc[2] += gJ00 * (-fx / (z * z)) + gJ11 * (-fy / (z * z));
        if (!G.clx) { gmc[0] += gJ02 * (-fx / (z * z)); gmc[2] += gJ02 * (2 * fx * x / (z * z * z)); }
        else { real lim = G.J[2] * z / -fx; gmc[2] += gJ02 * (fx * lim / (z * z)); }
        if (!G.cly) { gmc[1] += gJ12 * (-fy / (z * z)); gmc[2] += gJ12 * (2 * fy * y / (z * z * z)); }
        else { real lim = G.J[5] * z / -fy; gmc[2] += gJ12 * (fy * lim / (z * z)); }

        /* world mean: mu-hat = W mu + t */
        for (int j = 0; j < 3; j++) gm[j] += R[0 * 3 + j] * gmc[0] + R[1 * 3 + j] * gmc[1] + R[2 * 3 + j] * gmc[2];

        /* pose: d mu-hat = rho + phi x mu-hat ; dW = phi^ W                    */
        gp[0] += gmc[0]; gp[1] += gmc[1]; gp[2] += gmc[2];
        gp[3] += y * gmc[2] - z * gmc[1];
        gp[4] += z * gmc[0] - x * gmc[2];
        gp[5] += x * gmc[1] - y * gmc[0];
        real Pm[9];   /* W gW^T */
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                real s = 0;
                for (int k = 0; k < 3; k++) s += R[i * 3 + k] * gW[j * 3 + k];
                Pm[i * 3 + j] = s;
            }
        gp[3] += Pm[1 * 3 + 2] - Pm[2 * 3 + 1];
        gp[4] += Pm[2 * 3 + 0] - Pm[0 * 3 + 2];
        gp[5] += Pm[0 * 3 + 1] - Pm[1 * 3 + 0];
    }
    }
    for (int th = 0; th < nth; th++)
        for (int i = 0; i < 6; i++) g_pose[i] += pose_part[6 * th + i];
    free(pose_part);
}

/* ------------------------------------------------------------------------- */
/* Adam (bias-corrected), one parameter array.  Only entries with mask != 0  */
/* (or all, if mask is NULL) are updated; the rest keep p, m and v.          */
/* ------------------------------------------------------------------------- */
void orc_adam(int64_t count, int stride, const uint8_t* mask, real* p, real* m, real* v,
              const real* g, real lr, real b1, real b2, real eps, int64_t step)
{
    real bc1 = 1.0 - pow(b1, (real)step), bc2 = 1.0 - pow(b2, (real)step);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; i++) {
        if (mask && !mask[i / stride]) continue;
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        real mh = m[i] / bc1, vh = v[i] / bc2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ------------------------------------------------------------------------- */
/* Counter-based uniform generator: SplitMix64 (Steele, Lea, Flood 2014)     */
/* evaluated at counter i: mix(seed + (i+1) * golden-gamma); top 24 bits.    */
/* ------------------------------------------------------------------------- */
static uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double orc_uniform(uint64_t seed, uint64_t i)
{
    return (double)(splitmix64_at(seed, i) >> 40) * (1.0 / 16777216.0);
}

/* Sky Gaussians (§III-C 1): N_s points uniform by area on the upper         */
/* hemisphere (z >= 0) of radius R about the origin; scale = distance to the */
/* nearest other sky point (brute force).                                    */
void orc_sky(int64_t ns, double radius, uint64_t seed, float* xyz, double* nn_dist)
{
    for (int64_t i = 0; i < ns; i++) {
        double zc = orc_uniform(seed, 2 * (uint64_t)i);
        double ph = 2.0 * OR_PI * orc_uniform(seed, 2 * (uint64_t)i + 1);
        double rr = sqrt(1.0 - zc * zc);
        xyz[3 * i + 0] = (float)(radius * rr * cos(ph));
        xyz[3 * i + 1] = (float)(radius * rr * sin(ph));
        xyz[3 * i + 2] = (float)(radius * zc);
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < ns; i++) {
        double best = INFINITY;
        for (int64_t j = 0; j < ns; j++) {
            if (j == i) continue;
            double dx = (double)xyz[3 * i] - xyz[3 * j], dy = (double)xyz[3 * i + 1] - xyz[3 * j + 1];
            double dz = (double)xyz[3 * i + 2] - xyz[3 * j + 2];
            double d = dx * dx + dy * dy + dz * dz;
            if (d < best) best = d;
        }
        nn_dist[i] = sqrt(best);
    }
}

/* Map expansion (§III-C 2, Eq. 8): keep a point iff it projects (float32,   */
/* as the kernels decide) in front of z_near into the image and the opacity  */
/* map at its nearest pixel is below tau.  opacity == NULL keeps every point */
/* in front of z_near (the first frame).  Writes keep[i] and its depth.      */
int64_t orc_expand_mask(int64_t n, const float* xyz, const orc_cam* cam, const double* opacity,
                        double tau, uint8_t* keep, float* depth_f32)
{
    int64_t k = 0;
    float R[9], t[3];
    for (int i = 0; i < 9; i++) R[i] = (float)cam->R[i];
    for (int i = 0; i < 3; i++) t[i] = (float)cam->t[i];
    const float fx = (float)cam->fx, fy = (float)cam->fy, cx = (float)cam->cx, cy = (float)cam->cy;
    for (int64_t i = 0; i < n; i++) {
        const float* p = xyz + 3 * i;
        float x = ((R[0] * p[0] + R[1] * p[1]) + R[2] * p[2]) + t[0];
        float y = ((R[3] * p[0] + R[4] * p[1]) + R[5] * p[2]) + t[1];
        float z = ((R[6] * p[0] + R[7] * p[1]) + R[8] * p[2]) + t[2];
        depth_f32[i] = z;
        keep[i] = 0;
        if (!(z > OR_Z_NEAR_F)) continue;
        if (!opacity) { keep[i] = 1; k++; continue; }
        float iz = 1.0f / z;
        float u = fx * (x * iz) + cx;
        float v = fy * (y * iz) + cy;
        float pu = floorf(u + 0.5f), pv = floorf(v + 0.5f);
        if (!(pu >= 0.0f && pu < (float)cam->width && pv >= 0.0f && pv < (float)cam->height)) continue;
        size_t pix = (size_t)pv * cam->width + (size_t)pu;
        if (opacity[pix] < tau) { keep[i] = 1; k++; }
    }
    return k;
}
