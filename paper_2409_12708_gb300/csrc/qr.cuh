// qr.cuh -- batched blocked Householder QR, one CTA per matrix.
//
// A (m x n, column-major, leading dimension ld, in global memory) is factored
// as A = Q R with Q = H_0 H_1 ... H_{kk-1}, kk = min(m, n),
// H_j = I - tau_j v_j v_j^T, v_j(j) = 1, v_j(i < j) = 0 (Golub & Van Loan,
// Householder QR; the blocked form uses the compact WY representation
// H_0 ... H_{b-1} = I - V T V^T of Schreiber & Van Loan).  Panels of nb columns
// are factored in shared memory; the trailing columns are updated tile by tile
// through shared memory, so the matrix is read and written once per panel.
//
// Modes (after the factorisation):
//   QR_L_AND_Q : writes L = R^T (n x kk, row-major) and overwrites the first kk
//                columns of A with the thin Q (used to right-canonicalise a site:
//                A holds X^T, so X = L Q^T and Q^T becomes the site tensor).
//   QR_R_ROWS  : writes R (n x n, row-major, zero below the diagonal); m >= n.
#pragma once

#include "common.cuh"

namespace thc {

enum QRMode : int { QR_L_AND_Q = 1, QR_R_ROWS = 2 };

template <class T>
struct QRJob {
    T* A;          // term 0 matrix; term b at A + b * strideA
    long strideA;
    int m, n, ld;
    T* Tw;         // per-term panel T matrices, [ceil(kk/nb) * nb * nb]
    long strideT;
    T* out;        // L or R output
    long strideOut;
    int nb, tc;    // panel width, trailing tile width
    int mode;
    const int* colmap;  // optional per-term column permutation (n ints, stride n):
                        // logical column c is stored in physical column colmap[c]
};

__host__ __device__ inline int qr_ldp(int m) { return m | 1; }  // odd stride: conflict-free

#define QCOL(c) (cm ? cm[(c)] : (c))

constexpr int QR_THREADS = 512;  // 16 warps: one CTA per SM hides latency with more warps

__host__ __device__ inline int qr_gsize(int nb, int tc) { return nb * (tc > nb ? tc : nb); }

template <class T>
__host__ inline size_t qr_smem_bytes(int m, int nb, int tc) {
    return 64 * sizeof(double) + (size_t)(nb + tc) * qr_ldp(m) * sizeof(T) +
           (size_t)nb * nb * sizeof(T) + (size_t)qr_gsize(nb, tc) * sizeof(T) +
           (size_t)(QR_THREADS / 32) * 32 * tc * sizeof(T);
}

// Apply (H_p0 ... H_{p0+pw-1})^T (transpose=true, factorisation) or
// H_p0 ... H_{p0+pw-1} (transpose=false, forming Q) to columns [c_begin, c_end)
// of A, rows [p0, m).  P holds the panel's V (local rows, column i at
// P + i*ldp, unit diagonal implicit), Tm its T matrix.  Tiles of TC columns go
// through shared memory Y (column-major, stride ldp):
//   G = V^T Y : lane i of every warp owns row i of G (TC accumulators), the
//               warps split the rows of Y and their partial sums meet in Gp;
//   G <- T^T G (or T G), all threads, one column entry each;
//   Y -= V G  : each thread owns ROWS_PER_T rows of the tile and all TC columns.
constexpr int QR_TC = 8;

template <class T, int TC>
__device__ void qr_block_apply(T* A, int ld, int m, int p0, int pw, int c_begin, int c_end,
                               const T* P, int ldp, const T* Tm, int nbT, T* Y, T* G, T* Gp,
                               bool transpose, const int* cm) {
    const int R = m - p0;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int c0 = c_begin; c0 < c_end; c0 += TC) {
        const int tcn = min(TC, c_end - c0);
        for (int i = tid; i < TC * R; i += nt) {
            const int c = i / R, r = i % R;
            Y[c * ldp + r] = c < tcn ? A[(long)QCOL(c0 + c) * ld + p0 + r] : T(0);
        }
        __syncthreads();
        // partial G over this warp's rows
        {
            T acc[TC];
#pragma unroll
            for (int c = 0; c < TC; ++c) acc[c] = T(0);
            const int i = lane;
            if (i < pw) {
                const T* v = P + i * ldp;
                const int rs = ceil_div(R, nw);
                const int r0 = wid * rs, r1 = min(R, r0 + rs);
                for (int r = max(r0, i); r < r1; ++r) {
                    const T vr = (r == i) ? T(1) : v[r];
#pragma unroll
                    for (int c = 0; c < TC; ++c) acc[c] += vr * Y[c * ldp + r];
                }
            }
#pragma unroll
            for (int c = 0; c < TC; ++c) Gp[(wid * 32 + lane) * TC + c] = acc[c];
        }
        __syncthreads();
        for (int o = tid; o < pw * TC; o += nt) {
            const int i = o / TC, c = o % TC;
            T s = 0;
            for (int w = 0; w < nw; ++w) s += Gp[(w * 32 + i) * TC + c];
            G[i * TC + c] = s;
        }
        __syncthreads();
        // G <- T^T G (factorisation) or T G (forming Q); T upper triangular
        for (int o = tid; o < pw * TC; o += nt) {
            const int i = o / TC, c = o % TC;
            T s = 0;
            if (transpose) {
                for (int l = 0; l <= i; ++l) s += Tm[l * nbT + i] * G[l * TC + c];
            } else {
                for (int l = i; l < pw; ++l) s += Tm[i * nbT + l] * G[l * TC + c];
            }
            Gp[i * TC + c] = s;
        }
        __syncthreads();
        // Y -= V G, written straight back to A
        for (int r = tid; r < R; r += nt) {
            T acc[TC];
#pragma unroll
            for (int c = 0; c < TC; ++c) acc[c] = T(0);
            const int top = min(r, pw - 1);
            for (int l = 0; l <= top; ++l) {
                const T v = (l == r) ? T(1) : P[l * ldp + r];
#pragma unroll
                for (int c = 0; c < TC; ++c) acc[c] += v * Gp[l * TC + c];
            }
#pragma unroll
            for (int c = 0; c < TC; ++c)
                if (c < tcn) A[(long)QCOL(c0 + c) * ld + p0 + r] = Y[c * ldp + r] - acc[c];
        }
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(QR_THREADS) k_qr(QRJob<T> job) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = blockIdx.x;
    const int m = job.m, n = job.n, ld = job.ld, nb = job.nb, tc = job.tc;
    const int kk = min(m, n);
    const int ldp = qr_ldp(m);
    T* A = job.A + (long)b * job.strideA;
    T* Tw = job.Tw + (long)b * job.strideT;
    const int* cm = job.colmap ? job.colmap + (long)b * n : nullptr;
    double* red = reinterpret_cast<double*>(smem_raw);
    T* P = reinterpret_cast<T*>(smem_raw + 64 * sizeof(double));
    T* Y = P + (size_t)nb * ldp;
    T* Tm = Y + (size_t)tc * ldp;
    T* G = Tm + nb * nb;
    T* Gp = G + qr_gsize(nb, tc);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;

    for (int p0 = 0; p0 < kk; p0 += nb) {
        const int pw = min(nb, kk - p0);
        const int R = m - p0;
        for (int i = tid; i < pw * R; i += nt) {
            const int c = i / R, r = i % R;
            P[c * ldp + r] = A[(long)QCOL(p0 + c) * ld + p0 + r];
        }
        __syncthreads();
        // --- unblocked factorisation of the panel in shared memory
        for (int j = 0; j < pw; ++j) {
            T* x = P + j * ldp;
            // The squared norm is accumulated in float64: a reflector is orthogonal
            // only if beta^2 = alpha^2 + ||x||^2 holds to working precision, and a
            // float32 sum over ~10^3 entries misses that by ~1e-6, which then
            // compounds through the sweeps.
            double part = 0.0;
            for (int r = j + 1 + tid; r < R; r += nt) part += (double)x[r] * (double)x[r];
            const double xn2 = block_sum(part, red);
            // reflector parameters: one thread (float64), broadcast through shared memory
            if (tid == 0) {
                const double alpha = (double)x[j];
                double tau = 0.0, scale = 0.0;
                if (xn2 > 0.0) {
                    const double beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
                    tau = (beta - alpha) / beta;
                    scale = 1.0 / (alpha - beta);
                    x[j] = T(beta);
                }
                red[40] = tau;
                red[41] = scale;
                Tm[j * nb + j] = T(tau);
            }
            __syncthreads();
            const double tau = red[40];
            if (tau != 0.0) {
                const T scale = T(red[41]);
                for (int r = j + 1 + tid; r < R; r += nt) x[r] *= scale;
            }
            __syncthreads();
            // apply H_j^T to panel columns j+1 .. pw-1 (one warp per column)
            if (tau != 0.0) {
                for (int c = j + 1 + wid; c < pw; c += nw) {
                    T* y = P + c * ldp;
                    T s = 0;
                    for (int r = j + 1 + lane; r < R; r += 32) s += x[r] * y[r];
                    s = warp_sum(s) + y[j];
                    const T f = T(tau) * s;
                    if (lane == 0) y[j] -= f;
                    for (int r = j + 1 + lane; r < R; r += 32) y[r] -= f * x[r];
                }
            }
            __syncthreads();
        }
        // --- T matrix of the panel: T(0:j, j) = -tau_j T(0:j,0:j) V(:,0:j)^T v_j
        for (int o = tid; o < pw * pw; o += nt) {
            const int i = o / pw, j = o % pw;
            if (i < j) {
                const T* vi = P + i * ldp;
                const T* vj = P + j * ldp;
                T s = vi[j];
                for (int r = j + 1; r < R; ++r) s += vi[r] * vj[r];
                G[i * pw + j] = s;  // scratch: G holds at least nb*nb entries
            }
        }
        __syncthreads();
        // column j of T needs columns < j: one step per column, rows in parallel
        for (int j = 0; j < pw; ++j) {
            const T tj = Tm[j * nb + j];
            if (tid < j) {
                const int i = tid;
                T s = 0;
                for (int l = i; l < j; ++l) s += Tm[i * nb + l] * G[l * pw + j];
                Tm[i * nb + j] = -tj * s;
            } else if (tid > j && tid < pw) {
                Tm[tid * nb + j] = 0;
            }
            __syncthreads();
        }
        // keep T for forming Q; write the factored panel back
        for (int i = tid; i < nb * nb; i += nt) Tw[(p0 / nb) * nb * nb + i] = Tm[i];
        for (int i = tid; i < pw * R; i += nt) {
            const int c = i / R, r = i % R;
            A[(long)QCOL(p0 + c) * ld + p0 + r] = P[c * ldp + r];
        }
        __syncthreads();
        // --- trailing update of columns p0+pw .. n-1
        qr_block_apply<T, QR_TC>(A, ld, m, p0, pw, p0 + pw, n, P, ldp, Tm, nb, Y, G, Gp, true, cm);
    }

    // --- outputs
    T* out = job.out + (long)b * job.strideOut;
    if (job.mode == QR_R_ROWS) {
        for (int i = tid; i < n * n; i += nt) {
            const int r = i / n, c = i % n;
            out[i] = (r <= c && r < kk) ? A[(long)QCOL(c) * ld + r] : T(0);
        }
        return;
    }
    // QR_L_AND_Q: L = R^T (n x kk)
    for (int i = tid; i < n * kk; i += nt) {
        const int r = i / kk, c = i % kk;
        out[i] = (c <= r) ? A[(long)QCOL(r) * ld + c] : T(0);
    }
    __syncthreads();
    // form Q in place, panels in reverse order
    const int npan = ceil_div(kk, nb);
    for (int pi = npan - 1; pi >= 0; --pi) {
        const int p0 = pi * nb;
        const int pw = min(nb, kk - p0);
        const int R = m - p0;
        for (int i = tid; i < pw * R; i += nt) {
            const int c = i / R, r = i % R;
            P[c * ldp + r] = A[(long)QCOL(p0 + c) * ld + p0 + r];
        }
        for (int i = tid; i < nb * nb; i += nt) Tm[i] = Tw[pi * nb * nb + i];
        __syncthreads();
        if (p0 + pw < kk)
            qr_block_apply<T, QR_TC>(A, ld, m, p0, pw, p0 + pw, kk, P, ldp, Tm, nb, Y, G, Gp, false, cm);
        // panel columns in place (unblocked, backwards)
        for (int j = pw - 1; j >= 0; --j) {
            const T tj = Tm[j * nb + j];
            T* x = P + j * ldp;
            for (int c = j + 1 + wid; c < pw; c += nw) {
                T* y = P + c * ldp;
                T s = 0;
                for (int r = j + 1 + lane; r < R; r += 32) s += x[r] * y[r];
                s = warp_sum(s) + y[j];
                const T f = tj * s;
                if (lane == 0) y[j] -= f;
                for (int r = j + 1 + lane; r < R; r += 32) y[r] -= f * x[r];
            }
            __syncthreads();
            for (int r = j + 1 + tid; r < R; r += nt) x[r] = -tj * x[r];
            for (int r = tid; r < j; r += nt) x[r] = 0;
            if (tid == 0) x[j] = T(1) - tj;
            __syncthreads();
        }
        for (int i = tid; i < pw * m; i += nt) {
            const int c = i / m, r = i % m;
            A[(long)QCOL(p0 + c) * ld + r] = (r < p0) ? T(0) : P[c * ldp + (r - p0)];
        }
        __syncthreads();
    }
}

// Static column pivoting: perm[c] = index of the column with the c-th largest
// norm (ties by index).  Ordering the columns by norm before the Householder QR
// grades the rows of R, which cuts the number of one-sided Jacobi sweeps on R.
// One CTA per term; A column-major (m x n, ld); dynamic smem: n doubles.
template <class T>
__global__ void __launch_bounds__(256) k_colsort(const T* A, long strideA, int m, int n, int ld, int* perm) {
    extern __shared__ __align__(16) double cn[];
    const int b = blockIdx.x;
    A += (long)b * strideA;
    perm += (long)b * n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = wid; c < n; c += nw) {
        double acc = 0.0;
        for (int r = lane; r < m; r += 32) {
            const double x = A[(long)c * ld + r];
            acc += x * x;
        }
        acc = warp_sum(acc);
        if (lane == 0) cn[c] = acc;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const double v = cn[c];
        int rank = 0;
        for (int q = 0; q < n; ++q) rank += (cn[q] > v) || (cn[q] == v && q < c);
        perm[rank] = c;
    }
}

}  // namespace thc
