// qt_apply.cuh -- the SVD sweep's C_s = M_{s-1} Q_s without forming Q_s.
//
// The QR sweep leaves site s factored in place: X_s^T = Q R with the
// reflectors V below the diagonal of the m x kk column-major matrix A (unit
// diagonal implicit; R on and above it) and the compact-WY panel matrices T_p
// (Schreiber & Van Loan) in Tw.  The site tensor is the row-orthonormal
// Q^T = [I_kk 0] H_{kk-1} ... H_0 (real reflectors, H_j = H_j^T), so with
// P_p = H_{p0} ... H_{p0+pw-1} = I - V_p T_p V_p^T,
//     C = M Q^T = [M 0] P_{np-1}^T ... P_0^T,   P_p^T = I - V_p T_p^T V_p^T,
// applied from the last panel:  X <- X - (X V_p) T_p^T V_p^T,  X = [M 0].
// For out rows of M this is 4 out m kk flops, against 4 m kk^2 - 4 kk^3 / 3
// for forming Q plus 2 out m kk for the product M Q^T.
//
// One CTA of 512 threads per 32 rows of X (held in shared memory with a row
// pitch of m + 4 floats) and term:
//   * Z = X V_p: warp w takes a contiguous range of quads of the K = m - p0
//     rows of V_p; lane (rq, cq) accumulates the 8 x 4 tile rows rq + 4 i,
//     columns 4 cq.. with 16-byte loads of X (shared) and of V's columns
//     (global; the zero/one substitution of V's triangle only on the panel's
//     first 32 rows); the 16 warp partials are summed in shared memory;
//   * Z <- Z T_p^T (T upper triangular);
//   * X[:, p0:] -= Z V_p^T: two adjacent columns of X per thread, V's rows
//     k, k+1 read with one 8-byte load per panel column, coalesced across the
//     warp.
// Real float32 only, panels of 32 columns, m <= 1024 (the LQ-sweep shapes of
// the float paths up to D_max = 256); other shapes form Q in the QR kernel.
#pragma once

#include "common.cuh"

namespace thc {

constexpr int QT_THREADS = 512;
constexpr int QT_RB = 32;  // rows of X per CTA
constexpr int QT_NB = 32;  // panel width

template <class T>
struct QtJob {
    const T* M;   // out x kk rows, row-major, leading dimension ldM
    long strideM;
    int ldM;
    const T* A;   // m x kk reflectors, column-major, leading dimension ld
    long strideA;
    int ld;
    const T* Tw;  // panel p's T at Tw + p * QT_NB * QT_NB (row-major)
    long strideT;
    int out, m, kk;
    T* C;         // out x m result, row-major, leading dimension ldC
    long strideC;
    int ldC;
    T* W;         // optional column-major copy of C viewed as (4 out) x nW
    long strideW;
    int nW;
};

__host__ __device__ inline int qt_ldx(int m) { return m + 4; }

__host__ inline size_t qt_smem_bytes(int m) {
    return sizeof(float) * ((size_t)QT_RB * qt_ldx(m) + (size_t)(QT_THREADS / 32) * QT_RB * QT_NB +
                            2 * QT_RB * QT_NB + QT_NB * QT_NB);
}

// V_p's element (row k of A, panel column j): zero above the diagonal, one on it
__device__ __forceinline__ float qt_v(const float* A, int ld, int p0, int j, int k, float loaded) {
    const int kr = k - p0;
    return kr < j ? 0.f : (kr == j ? 1.f : loaded);
}

static __global__ void __launch_bounds__(QT_THREADS, 1) k_apply_qt(QtJob<float> job) {
    extern __shared__ __align__(16) unsigned char qt_raw[];
    const int b = blockIdx.y, r0 = blockIdx.x * QT_RB;
    const int m = job.m, kk = job.kk, ldx = qt_ldx(m);
    const int rows = min(QT_RB, job.out - r0);
    float* X = reinterpret_cast<float*>(qt_raw);                 // QT_RB x ldx
    float* Zp = X + (size_t)QT_RB * ldx;                          // 16 warps x (QT_RB x QT_NB)
    float* Z = Zp + (size_t)(QT_THREADS / 32) * QT_RB * QT_NB;    // QT_RB x QT_NB
    float* Z2 = Z + QT_RB * QT_NB;                                // Z T^T
    float* Tm = Z2 + QT_RB * QT_NB;                               // QT_NB x QT_NB
    const float* M = job.M + (long)b * job.strideM;
    const float* A = job.A + (long)b * job.strideA;
    const float* Tw = job.Tw + (long)b * job.strideT;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = QT_THREADS / 32;
    for (int r = 0; r < QT_RB; ++r)
        for (int c = tid; c < m; c += QT_THREADS)
            X[(size_t)r * ldx + c] = (r < rows && c < kk) ? M[(long)(r0 + r) * job.ldM + c] : 0.f;
    // tile of lane (rq, cq): rows rq + 4 i (i < 8), columns 4 cq .. 4 cq + 3; the
    // four rows a quarter-warp reads together are consecutive, and the pitch
    // m + 4 puts them in distinct bank quads
    const int rq = lane >> 3, cq = lane & 7;
    const int np = ceil_div(kk, QT_NB);
    for (int p = np - 1; p >= 0; --p) {
        const int p0 = p * QT_NB, pw = min(QT_NB, kk - p0);
        for (int i = tid; i < QT_NB * QT_NB; i += QT_THREADS) Tm[i] = Tw[(long)p * QT_NB * QT_NB + i];
        __syncthreads();
        // ---- Z = X[:, p0:m] V_p, K split over the warps in quads of rows
        {
            const int R4 = (m - p0) >> 2;  // m and p0 are multiples of 4
            const int qpw = ceil_div(R4, nw);
            const int q0 = wid * qpw, q1 = min(R4, q0 + qpw);
            float acc[8][4];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
            for (int q = q0; q < q1; ++q) {
                const int k = p0 + 4 * q;
                float4 v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int col = 4 * cq + j;
                    v[j] = col < pw ? *reinterpret_cast<const float4*>(A + (long)(p0 + col) * job.ld + k)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                if (k < p0 + QT_NB) {  // the panel's triangle: zeros above the diagonal, ones on it
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int col = 4 * cq + j;
                        v[j] = make_float4(qt_v(A, job.ld, p0, col, k, v[j].x), qt_v(A, job.ld, p0, col, k + 1, v[j].y),
                                           qt_v(A, job.ld, p0, col, k + 2, v[j].z),
                                           qt_v(A, job.ld, p0, col, k + 3, v[j].w));
                    }
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float4 x = *reinterpret_cast<const float4*>(X + (size_t)(rq + 4 * i) * ldx + k);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float a = acc[i][j];
                        a = fmaf(x.x, v[j].x, a);
                        a = fmaf(x.y, v[j].y, a);
                        a = fmaf(x.z, v[j].z, a);
                        acc[i][j] = fmaf(x.w, v[j].w, a);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    Zp[(size_t)wid * QT_RB * QT_NB + (rq + 4 * i) * QT_NB + 4 * cq + j] = acc[i][j];
        }
        __syncthreads();
        for (int o = tid; o < QT_RB * QT_NB; o += QT_THREADS) {
            float s = 0.f;
            for (int w = 0; w < nw; ++w) s += Zp[(size_t)w * QT_RB * QT_NB + o];
            Z[o] = s;
        }
        __syncthreads();
        // ---- Z2 = Z T^T: Z2(r, j) = sum_{i >= j} Z(r, i) T(j, i)
        for (int o = tid; o < QT_RB * QT_NB; o += QT_THREADS) {
            const int r = o / QT_NB, j = o - r * QT_NB;
            float s = 0.f;
            if (j < pw)
                for (int i = j; i < pw; ++i) s += Z[r * QT_NB + i] * Tm[j * QT_NB + i];
            Z2[o] = s;
        }
        __syncthreads();
        // ---- X[:, p0:m] -= Z2 V_p^T, two adjacent columns per thread (p0 and m
        // are even): V's rows k, k+1 come with one 8-byte load per panel column
        for (int k = p0 + 2 * tid; k < m; k += 2 * QT_THREADS) {
            float2 v[QT_NB];
#pragma unroll
            for (int j = 0; j < QT_NB; ++j)
                v[j] = j < pw ? *reinterpret_cast<const float2*>(A + (long)(p0 + j) * job.ld + k)
                              : make_float2(0.f, 0.f);
            if (k < p0 + QT_NB) {  // the panel's triangle
#pragma unroll
                for (int j = 0; j < QT_NB; ++j) {
                    v[j].x = qt_v(A, job.ld, p0, j, k, v[j].x);
                    v[j].y = qt_v(A, job.ld, p0, j, k + 1, v[j].y);
                }
            }
#pragma unroll 2
            for (int r = 0; r < QT_RB; ++r) {
                const float4* zr = reinterpret_cast<const float4*>(Z2 + r * QT_NB);
                float s0 = 0.f, s1 = 0.f;
#pragma unroll
                for (int j4 = 0; j4 < QT_NB / 4; ++j4) {
                    const float4 z = zr[j4];
                    s0 = fmaf(z.x, v[4 * j4].x, s0);
                    s1 = fmaf(z.x, v[4 * j4].y, s1);
                    s0 = fmaf(z.y, v[4 * j4 + 1].x, s0);
                    s1 = fmaf(z.y, v[4 * j4 + 1].y, s1);
                    s0 = fmaf(z.z, v[4 * j4 + 2].x, s0);
                    s1 = fmaf(z.z, v[4 * j4 + 2].y, s1);
                    s0 = fmaf(z.w, v[4 * j4 + 3].x, s0);
                    s1 = fmaf(z.w, v[4 * j4 + 3].y, s1);
                }
                float2* xr = reinterpret_cast<float2*>(X + (size_t)r * ldx + k);
                float2 x = *xr;
                x.x -= s0;
                x.y -= s1;
                *xr = x;
            }
        }
        __syncthreads();
    }
    // ---- C (and its column-major copy for the preconditioning QR)
    float* C = job.C + (long)b * job.strideC;
    for (int r = 0; r < rows; ++r)
        for (int c = tid; c < m; c += QT_THREADS) C[(long)(r0 + r) * job.ldC + c] = X[(size_t)r * ldx + c];
    if (job.W) {
        // W viewed as (4 out) x nW column-major; m = 4 nW
        float* W = job.W + (long)b * job.strideW;
        const int mW = 4 * job.out;
        for (int r = 0; r < rows; ++r)
            for (int qb = 0; qb < 4; ++qb)
                for (int j = tid; j < job.nW; j += QT_THREADS)
                    W[(long)j * mW + (r0 + r) * 4 + qb] = X[(size_t)r * ldx + qb * job.nW + j];
    }
}

}  // namespace thc
