// qr.cuh -- batched blocked Householder QR, one CTA per matrix.
//
// A (m x n, column-major, leading dimension ld, in global memory) is factored
// as A = Q R with Q = H_0 H_1 ... H_{kk-1}, kk = min(m, n),
// H_j = I - tau_j v_j v_j^T, v_j(j) = 1, v_j(i < j) = 0 (Golub & Van Loan,
// Householder QR; the blocked form uses the compact WY representation
// H_0 ... H_{b-1} = I - V T V^T of Schreiber & Van Loan).  Panels of nb columns
// are factored in shared memory; the trailing columns are updated in groups of
// QR_QG columns straight from global memory with register-tiled products
// (W = V^T Y, W <- T^T W, Y -= V W), so each group is read twice and written
// once per panel.
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
    int nb;        // panel width
    int mode;
    const int* colmap;  // optional per-term column permutation (n ints, stride n):
                        // logical column c is stored in physical column colmap[c]
};

// physical column of logical column c under the optional column map cm
#define QCOL(c) (cm ? cm[(c)] : (c))

constexpr int QR_THREADS = 512;  // 16 warps: one CTA per SM hides latency with more warps
constexpr int QR_QG = 16;        // trailing columns per group

// Column stride of the panel in shared memory: a multiple of 16 bytes (vector
// access to 4 consecutive rows) that is 16 bytes past a multiple of 128, so
// the columns a warp reads at once fall in distinct bank groups.
template <class T>
__host__ __device__ inline int qr_ldp(int m) {
    return sizeof(T) == 4 ? (m + 31) / 32 * 32 + 4 : (m + 15) / 16 * 16 + 2;
}

// Reflector rows per lane in the register-tiled products (lane (ig, cg) owns
// rows ig + 8 ii of W, ii < qr_ni(nb), and columns 4 cg .. 4 cg + 3).
__host__ __device__ inline int qr_ni(int nb) { return nb >= 32 ? 4 : (nb >= 16 ? 2 : 1); }

template <class T>
__host__ inline size_t qr_smem_bytes(int m, int nb) {
    const size_t cap = 8 * qr_ni(nb);  // rows of W per warp partial
    return 64 * sizeof(double) + (size_t)nb * qr_ldp<T>(m) * sizeof(T) + 2 * (size_t)nb * nb * sizeof(T) +
           ((size_t)(QR_THREADS / 32) * cap * QR_QG + 2 * cap * QR_QG) * sizeof(T);
}

// four consecutive elements with 16-byte accesses (p 16-byte aligned)
template <class T>
__device__ __forceinline__ void ld4(T (&x)[4], const T* p) {
    if constexpr (sizeof(T) == 4) {
        const float4 u = *reinterpret_cast<const float4*>(p);
        x[0] = u.x;
        x[1] = u.y;
        x[2] = u.z;
        x[3] = u.w;
    } else {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 b = *reinterpret_cast<const double2*>(p + 2);
        x[0] = a.x;
        x[1] = a.y;
        x[2] = b.x;
        x[3] = b.y;
    }
}
template <class T>
__device__ __forceinline__ void st4(T* p, const T (&x)[4]) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    } else {
        *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
        *reinterpret_cast<double2*>(p + 2) = make_double2(x[2], x[3]);
    }
}
// rows r .. r+3 of a global column (zeros at or beyond R); vector access when allowed
template <class T>
__device__ __forceinline__ void ld4_col(T (&x)[4], const T* col, int r, int R, bool vec) {
    if (vec && r + 4 <= R) {
        ld4(x, col + r);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = r + q < R ? col[r + q] : T(0);
    }
}
template <class T>
__device__ __forceinline__ void st4_col(T* col, const T (&x)[4], int r, int R, bool vec) {
    if (vec && r + 4 <= R) {
        st4(col + r, x);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (r + q < R) col[r + q] = x[q];
    }
}

// Apply (H_p0 ... H_{p0+pw-1})^T (transpose=true, factorisation) or
// H_p0 ... H_{p0+pw-1} (transpose=false, forming Q) to columns [c_begin, c_end)
// of A, rows [p0, m).  P holds the panel's V explicitly (column i at
// P + i*ldp: zeros above row i, 1 at row i, zero rows from R up to the next
// multiple of 4); Tm its T matrix.  Per group of QR_QG columns:
//   W_w = V^T Y over the rows of warp w (lane (ig, cg): rows ig + 8 ii of W,
//         columns 4 cg .. 4 cg + 3; four rows of Y per step), summed into W0;
//   W1  = T^T W0 (or T W0);
//   Y  -= V W1, each thread a tile of 4 rows x 4 columns.
// Every product step is 16-byte loads and an outer-product of 4-vectors.
template <class T, int NI>
__device__ void qr_block_apply(T* A, int ld, int m, int p0, int pw, int c_begin, int c_end, const T* P, int ldp,
                               const T* Tm, int nbT, T* Wp, T* W0, T* W1, bool transpose, const int* cm,
                               bool vec) {
    constexpr int CAP = 8 * NI;
    const int R = m - p0;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    const int ig = lane >> 2, cg = lane & 3;
    const int R4 = ceil_div(R, 4);
    const int qpw = ceil_div(R4, nw);
    const int r0 = 4 * wid * qpw, r1 = min(R, 4 * (wid + 1) * qpw);
    for (int c0 = c_begin; c0 < c_end; c0 += QR_QG) {
        {
            T acc[NI][4];
#pragma unroll
            for (int ii = 0; ii < NI; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = T(0);
            const T* yc[4];
            bool cok[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int col = c0 + 4 * cg + jj;
                cok[jj] = col < c_end;
                yc[jj] = A + (long)QCOL(cok[jj] ? col : c0) * ld + p0;
            }
            for (int r = r0; r < r1; r += 4) {
                T v[NI][4], y[4][4];
#pragma unroll
                for (int ii = 0; ii < NI; ++ii) {
                    if (ig + 8 * ii < pw) {
                        ld4(v[ii], P + (ig + 8 * ii) * ldp + r);
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) v[ii][q] = T(0);
                    }
                }
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    if (cok[jj]) {
                        ld4_col(y[jj], yc[jj], r, R, vec);
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) y[jj][q] = T(0);
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int ii = 0; ii < NI; ++ii)
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) acc[ii][jj] += v[ii][q] * y[jj][q];
            }
#pragma unroll
            for (int ii = 0; ii < NI; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) Wp[(wid * CAP + ig + 8 * ii) * QR_QG + 4 * cg + jj] = acc[ii][jj];
        }
        __syncthreads();
        for (int o = tid; o < pw * QR_QG; o += nt) {
            T s = 0;
            for (int w = 0; w < nw; ++w) s += Wp[w * CAP * QR_QG + o];
            W0[o] = s;
        }
        __syncthreads();
        // W1 = T^T W0 (factorisation) or T W0 (forming Q); T upper triangular
        for (int o = tid; o < pw * QR_QG; o += nt) {
            const int i = o / QR_QG, c = o % QR_QG;
            T s = 0;
            if (transpose) {
                for (int l = 0; l <= i; ++l) s += Tm[l * nbT + i] * W0[l * QR_QG + c];
            } else {
                for (int l = i; l < pw; ++l) s += Tm[i * nbT + l] * W0[l * QR_QG + c];
            }
            W1[o] = s;
        }
        __syncthreads();
        // Y -= V W1 (consecutive threads take consecutive row quads of a column quad)
        const int ncq = ceil_div(min(QR_QG, c_end - c0), 4);
        for (int t = tid; t < R4 * ncq; t += nt) {
            const int cq = t / R4, r = 4 * (t - cq * R4);
            T* yc[4];
            bool cok[4];
            T y[4][4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int col = c0 + 4 * cq + jj;
                cok[jj] = col < c_end;
                yc[jj] = A + (long)QCOL(cok[jj] ? col : c0) * ld + p0;
                if (cok[jj]) {
                    ld4_col(y[jj], yc[jj], r, R, vec);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) y[jj][q] = T(0);
                }
            }
            T acc[4][4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[jj][q] = T(0);
#pragma unroll 4
            for (int i = 0; i < pw; ++i) {
                T vq[4], w[4];
                ld4(vq, P + i * ldp + r);
                ld4(w, W1 + i * QR_QG + 4 * cq);
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[jj][q] += vq[q] * w[jj];
            }
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
#pragma unroll
                for (int q = 0; q < 4; ++q) y[jj][q] -= acc[jj][q];
                if (cok[jj]) st4_col(yc[jj], y[jj], r, R, vec);
            }
        }
        __syncthreads();
    }
}

template <class T>
__device__ __forceinline__ void qr_block_apply_nb(T* A, int ld, int m, int p0, int pw, int c_begin, int c_end,
                                                  const T* P, int ldp, const T* Tm, int nbT, T* Wp, T* W0, T* W1,
                                                  bool transpose, const int* cm, bool vec) {
    const int ni = qr_ni(nbT);
    if (ni == 4)
        qr_block_apply<T, 4>(A, ld, m, p0, pw, c_begin, c_end, P, ldp, Tm, nbT, Wp, W0, W1, transpose, cm, vec);
    else if (ni == 2)
        qr_block_apply<T, 2>(A, ld, m, p0, pw, c_begin, c_end, P, ldp, Tm, nbT, Wp, W0, W1, transpose, cm, vec);
    else
        qr_block_apply<T, 1>(A, ld, m, p0, pw, c_begin, c_end, P, ldp, Tm, nbT, Wp, W0, W1, transpose, cm, vec);
}

// Panel in shared memory as explicit V: zeros above the diagonal, 1 on it.
template <class T>
__device__ __forceinline__ void qr_explicit_v(T* P, int ldp, int pw) {
    for (int o = threadIdx.x; o < pw * pw; o += blockDim.x) {
        const int i = o / pw, r = o % pw;  // column i, row r
        if (r <= i) P[i * ldp + r] = (r == i) ? T(1) : T(0);
    }
}

template <class T>
__global__ void __launch_bounds__(QR_THREADS) k_qr(QRJob<T> job) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = blockIdx.x;
    const int m = job.m, n = job.n, ld = job.ld, nb = job.nb;
    const int kk = min(m, n);
    const int ldp = qr_ldp<T>(m);
    T* A = job.A + (long)b * job.strideA;
    T* Tw = job.Tw + (long)b * job.strideT;
    const int* cm = job.colmap ? job.colmap + (long)b * n : nullptr;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    const int cap = 8 * qr_ni(nb);
    double* red = reinterpret_cast<double*>(smem_raw);
    T* P = reinterpret_cast<T*>(smem_raw + 64 * sizeof(double));
    T* Tm = P + (size_t)nb * ldp;
    T* G = Tm + nb * nb;
    T* Wp = G + nb * nb;
    T* W0 = Wp + (size_t)nw * cap * QR_QG;
    T* W1 = W0 + (size_t)cap * QR_QG;
    // 16-byte accesses to columns of A (rows p0 + r, r a multiple of 4)
    const bool vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (ld % 4 == 0);

    for (int p0 = 0; p0 < kk; p0 += nb) {
        const int pw = min(nb, kk - p0);
        const int R = m - p0;
        const int R4 = 4 * ceil_div(R, 4);
        for (int i = tid; i < pw * R4; i += nt) {
            const int c = i / R4, r = i % R4;
            P[c * ldp + r] = r < R ? A[(long)QCOL(p0 + c) * ld + p0 + r] : T(0);
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
        if (p0 + pw < n) {
            qr_explicit_v(P, ldp, pw);
            __syncthreads();
            qr_block_apply_nb<T>(A, ld, m, p0, pw, p0 + pw, n, P, ldp, Tm, nb, Wp, W0, W1, true, cm, vec);
        }
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
        const int R4 = 4 * ceil_div(R, 4);
        for (int i = tid; i < pw * R4; i += nt) {
            const int c = i / R4, r = i % R4;
            P[c * ldp + r] = r < R ? A[(long)QCOL(p0 + c) * ld + p0 + r] : T(0);
        }
        for (int i = tid; i < nb * nb; i += nt) Tm[i] = Tw[pi * nb * nb + i];
        __syncthreads();
        qr_explicit_v(P, ldp, pw);
        __syncthreads();
        if (p0 + pw < kk)
            qr_block_apply_nb<T>(A, ld, m, p0, pw, p0 + pw, kk, P, ldp, Tm, nb, Wp, W0, W1, false, cm, vec);
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
