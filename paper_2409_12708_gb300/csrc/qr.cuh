// qr.cuh -- batched blocked Householder QR, one CTA per matrix.
//
// A (m x n, column-major, leading dimension ld, in global memory) is factored
// as A = Q R with Q = H_0 H_1 ... H_{kk-1}, kk = min(m, n),
// H_j = I - tau_j v_j v_j^H, v_j(j) = 1, v_j(i < j) = 0 (Golub & Van Loan,
// Householder QR; for complex A the reflector of LAPACK's convention, with a
// real beta and a complex tau, and H_j^H applied to the trailing columns; the
// blocked form uses the compact WY representation H_0 ... H_{b-1} =
// I - V T V^H of Schreiber & Van Loan).  Panels of nb columns are factored in
// shared memory; the trailing columns are updated in groups of QR_QG columns
// straight from global memory with register-tiled products
// (W = V^H Y, W <- T^H W, Y -= V W), so each group is read twice and written
// once per panel.  Real and complex scalars share the code (scalar.cuh).
//
// Modes (after the factorisation):
//   QR_L_AND_Q : writes L = R^T (n x kk, row-major) and overwrites the first kk
//                columns of A with the thin Q (used to right-canonicalise a site:
//                A holds X^T, so X = L Q^T and Q^T becomes the site tensor; for
//                complex X the plain transpose keeps Q^T's rows orthonormal).
//   QR_R_ROWS  : writes R (n x n, row-major, zero below the diagonal); m >= n.
//   QR_L_ONLY  : writes L as QR_L_AND_Q and leaves the reflectors in A and the
//                panel T matrices in Tw (Q is applied later without being formed).
#pragma once

#include "common.cuh"
#include "scalar.cuh"

namespace thc {

enum QRMode : int { QR_L_AND_Q = 1, QR_R_ROWS = 2, QR_L_ONLY = 3 };

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
    int* colmap;   // optional per-term column permutation (n ints, stride n):
                   // logical column c is stored in physical column colmap[c]
    int pivot;     // QR_R_ROWS only: choose the column order by block pivoting
                   // (colmap is then an output: the chosen order)
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
    constexpr int e16 = 16 / (int)sizeof(T), e128 = 128 / (int)sizeof(T);
    return (m + e128 - 1) / e128 * e128 + e16;
}

// Reflector rows per lane in the register-tiled products (lane (ig, cg) owns
// rows ig + 8 ii of W, ii < qr_ni(nb), and columns 4 cg .. 4 cg + 3).
__host__ __device__ inline int qr_ni(int nb) { return nb >= 32 ? 4 : (nb >= 16 ? 2 : 1); }

template <class T>
__host__ inline size_t qr_smem_bytes(int m, int nb, int n) {
    const size_t cap = 8 * qr_ni(nb);  // rows of W per warp partial
    const size_t base = 64 * sizeof(double) + (size_t)nb * qr_ldp<T>(m) * sizeof(T) + 2 * (size_t)nb * nb * sizeof(T) +
                        ((size_t)(QR_THREADS / 32) * cap * QR_QG + 2 * cap * QR_QG) * sizeof(T);
    // pivoting state: nb float64 norms, nb + n (real) metrics / norms, two n-int column maps
    const size_t piv = (size_t)nb * sizeof(double) + (size_t)(nb + n) * sizeof(real_t<T>) +
                       2 * (size_t)n * sizeof(int);
    return base + ((piv + 15) & ~(size_t)15);
}

// four consecutive elements with 16-byte accesses (p 16-byte aligned)
template <class T>
__device__ __forceinline__ void ld4(T (&x)[4], const T* p) {
    if constexpr (is_complex_v<T>) {
        constexpr int NV = 4 * (int)sizeof(T) / 16;  // 16-byte words
        uint4 u[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) u[q] = reinterpret_cast<const uint4*>(p)[q];
        const T* pu = reinterpret_cast<const T*>(u);
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = pu[q];
    } else if constexpr (sizeof(T) == 4) {
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
    if constexpr (is_complex_v<T>) {
        constexpr int NV = 4 * (int)sizeof(T) / 16;
        uint4 u[NV];
        T* pu = reinterpret_cast<T*>(u);
#pragma unroll
        for (int q = 0; q < 4; ++q) pu[q] = x[q];
#pragma unroll
        for (int q = 0; q < NV; ++q) reinterpret_cast<uint4*>(p)[q] = u[q];
    } else if constexpr (sizeof(T) == 4) {
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
        for (int q = 0; q < 4; ++q) x[q] = r + q < R ? col[r + q] : tzero<T>();
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

// Squared norm with about twice the storage precision.  A Householder
// reflector is orthogonal only if beta^2 = alpha^2 + ||x||^2 holds to working
// precision, and a plain float32 sum over ~10^3 entries misses that by ~1e-6,
// which then compounds through the sweeps.  float: float-float accumulation
// (Knuth's TwoSum with the exact product error from an FMA), no float64
// arithmetic on the hot path; double: a plain sum.
template <class T>
struct SqAcc;
template <>
struct SqAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x * x; }
    __device__ __forceinline__ double warp_total() { return warp_sum(s); }
};
template <>
struct SqAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float p = x * x, e = fmaf(x, x, -p);
        const float s = hi + p, bp = s - hi;
        lo += ((hi - (s - bp)) + (p - bp)) + e;
        hi = s;
    }
    // butterfly of float-float pairs; every lane ends with the same total
    __device__ __forceinline__ double warp_total() {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
            const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            const float s = hi + h2, bp = s - hi;
            lo = (lo + l2) + ((hi - (s - bp)) + (h2 - bp));
            hi = s;
        }
        return (double)hi + (double)lo;
    }
};

// complex: both parts of every entry go through the accumulator of the real type
template <class R>
struct SqAcc<cplx<R>> {
    SqAcc<R> a;
    __device__ __forceinline__ void add(cplx<R> x) {
        a.add(x.x);
        a.add(x.y);
    }
    __device__ __forceinline__ double warp_total() { return a.warp_total(); }
};

// |x|^2 evaluated in float64
template <class T>
__device__ __forceinline__ double dabs2(T x) {
    if constexpr (is_complex_v<T>) return (double)x.x * (double)x.x + (double)x.y * (double)x.y;
    else return (double)x * (double)x;
}

// Squared norm of y[r0 .. R) by one warp (every lane gets the total).  In
// float32, squares of entries below ~1e-19 underflow or lose their precision
// (residues of rank-deficient columns are of that size), which would make the
// reflector inconsistent with its vector; such small totals are recomputed
// from float64 squares.
template <class T>
__device__ __forceinline__ double col_norm2(const T* y, int r0, int R) {
    const int lane = threadIdx.x & 31;
    SqAcc<T> a;
    for (int r = r0 + lane; r < R; r += 32) a.add(y[r]);
    double t = a.warp_total();
    if (sizeof(real_t<T>) == 4 && t < 1e-30) {
        double s = 0.0;
        for (int r = r0 + lane; r < R; r += 32) s += dabs2(y[r]);
        t = warp_sum(s);
    }
    return t;
}

// Register-tiled pieces of the compact-WY update with the panel's V held
// explicitly in shared memory (column i at P + i*ldp: zeros above row i, 1 at
// row i, zero rows from R up to the next multiple of 4).
//
// (1) Per-warp partial products Wp[w] = V^H Y over the rows of warp w for the
//     QR_QG columns whose bases col(c) returns (c < QR_QG; null: no column).
//     Lane (ig, cg) owns rows ig + 8 ii of W and columns 4 cg .. 4 cg + 3; each
//     step takes four rows of V and Y with 16-byte loads.
template <class T, int NI, class ColF>
__device__ __forceinline__ void qr_vty(const T* P, int ldp, int pw, int R, T* Wp, ColF col, bool vec) {
    constexpr int CAP = 8 * NI;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ig = lane >> 2, cg = lane & 3;
    const int R4 = ceil_div(R, 4), qpw = ceil_div(R4, nw);
    const int r0 = 4 * wid * qpw, r1 = min(R, 4 * (wid + 1) * qpw);
    T acc[NI][4];
#pragma unroll
    for (int ii = 0; ii < NI; ++ii)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = tzero<T>();
    const T* yc[4];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) yc[jj] = col(4 * cg + jj);
    for (int r = r0; r < r1; r += 4) {
        T v[NI][4], y[4][4];
#pragma unroll
        for (int ii = 0; ii < NI; ++ii) {
            if (ig + 8 * ii < pw) {
                ld4(v[ii], P + (ig + 8 * ii) * ldp + r);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[ii][q] = tzero<T>();
            }
        }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            if (yc[jj]) {
                ld4_col(y[jj], yc[jj], r, R, vec);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) y[jj][q] = tzero<T>();
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int ii = 0; ii < NI; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[ii][jj] += tconj_mul(v[ii][q], y[jj][q]);
    }
#pragma unroll
    for (int ii = 0; ii < NI; ++ii)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) Wp[(wid * CAP + ig + 8 * ii) * QR_QG + 4 * cg + jj] = acc[ii][jj];
}

// (2) W0 = sum of the warp partials (pw x QR_QG)
template <class T>
__device__ __forceinline__ void qr_sum_partials(const T* Wp, T* W0, int pw, int cap) {
    const int nw = blockDim.x >> 5;
    for (int o = threadIdx.x; o < pw * QR_QG; o += blockDim.x) {
        T s = tzero<T>();
        for (int w = 0; w < nw; ++w) s += Wp[w * cap * QR_QG + o];
        W0[o] = s;
    }
}

// (3) W1 = T^H W0 (factorisation) or T W0 (forming Q); T upper triangular
template <class T>
__device__ __forceinline__ void qr_t_times(const T* Tm, int nbT, const T* W0, T* W1, int pw, bool transpose) {
    for (int o = threadIdx.x; o < pw * QR_QG; o += blockDim.x) {
        const int i = o / QR_QG, c = o % QR_QG;
        T s = tzero<T>();
        if (transpose) {
            for (int l = 0; l <= i; ++l) s += tconj_mul(Tm[l * nbT + i], W0[l * QR_QG + c]);
        } else {
            for (int l = i; l < pw; ++l) s += Tm[i * nbT + l] * W0[l * QR_QG + c];
        }
        W1[o] = s;
    }
}

// (4) Y -= V W1 for ncols (<= QR_QG) columns, each thread a tile of 4 rows x 4
//     columns (consecutive threads: consecutive row quads of a column quad).
//     col(c) gives the base of column c in global memory.  IDENT: Y starts as
//     the identity columns (local row cb + c of column c is 1) instead of
//     being loaded.
template <class T, bool IDENT, class ColF>
__device__ __forceinline__ void qr_sub_vw(const T* P, int ldp, int pw, int R, const T* W1, int ncols, int cb,
                                          ColF col, bool vec) {
    const int R4 = ceil_div(R, 4), ncq = ceil_div(ncols, 4);
    for (int t = threadIdx.x; t < R4 * ncq; t += blockDim.x) {
        const int cq = t / R4, r = 4 * (t - cq * R4);
        T* yc[4];
        T y[4][4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int c = 4 * cq + jj;
            yc[jj] = c < ncols ? col(c) : nullptr;
            if (IDENT) {
#pragma unroll
                for (int q = 0; q < 4; ++q) y[jj][q] = (r + q == cb + c) ? tone<T>() : tzero<T>();
            } else if (yc[jj]) {
                ld4_col(y[jj], yc[jj], r, R, vec);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) y[jj][q] = tzero<T>();
            }
        }
        T acc[4][4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[jj][q] = tzero<T>();
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
            if (yc[jj]) st4_col(yc[jj], y[jj], r, R, vec);
        }
    }
}

// Apply (H_p0 ... H_{p0+pw-1})^H (transpose=true, factorisation) or
// H_p0 ... H_{p0+pw-1} (transpose=false, forming Q) to columns [c_begin, c_end)
// of A, rows [p0, m), in groups of QR_QG columns: W = V^H Y, W <- T^H W (or
// T W), Y -= V W.  Every product step is 16-byte loads and an outer product
// of 4-vectors.
template <class T, int NI>
__device__ void qr_block_apply(T* A, int ld, int m, int p0, int pw, int c_begin, int c_end, const T* P, int ldp,
                               const T* Tm, int nbT, T* Wp, T* W0, T* W1, bool transpose, const int* cm,
                               bool vec) {
    const int R = m - p0;
    for (int c0 = c_begin; c0 < c_end; c0 += QR_QG) {
        auto col = [&](int c) -> T* {
            const int cc = c0 + c;
            return cc < c_end ? A + (long)QCOL(cc) * ld + p0 : nullptr;
        };
        qr_vty<T, NI>(P, ldp, pw, R, Wp, col, vec);
        __syncthreads();
        qr_sum_partials(Wp, W0, pw, 8 * NI);
        __syncthreads();
        qr_t_times(Tm, nbT, W0, W1, pw, transpose);
        __syncthreads();
        qr_sub_vw<T, false>(P, ldp, pw, R, W1, min(QR_QG, c_end - c0), 0, col, vec);
        __syncthreads();
    }
}

// Columns p0 .. p0+pw-1 of Q = H_0 ... H_{kk-1} [I; 0] once the later panels
// are applied: rows p0.. of those columns are H_p0 ... H_{p0+pw-1} E with E the
// identity columns, i.e. E - V (T V1^H) with V1 the top pw x pw block of V
// (V^H E = V1^H); rows above p0 are zero.
template <class T>
__device__ void qr_form_panel(T* A, int ld, int m, int p0, int pw, const T* P, int ldp, const T* Tm, int nbT,
                              T* W0, T* W1, const int* cm, bool vec) {
    const int R = m - p0;
    for (int cb = 0; cb < pw; cb += QR_QG) {
        const int gc = min(QR_QG, pw - cb);
        for (int o = threadIdx.x; o < pw * QR_QG; o += blockDim.x) {
            const int i = o / QR_QG, c = o % QR_QG;
            W0[o] = c < gc ? tconj(P[i * ldp + cb + c]) : tzero<T>();
        }
        __syncthreads();
        qr_t_times(Tm, nbT, W0, W1, pw, false);
        __syncthreads();
        auto col = [&](int c) -> T* { return A + (long)QCOL(p0 + cb + c) * ld + p0; };
        qr_sub_vw<T, true>(P, ldp, pw, R, W1, gc, cb, col, vec);
        __syncthreads();
    }
    for (int i = threadIdx.x; i < pw * p0; i += blockDim.x) {
        const int c = i / p0, r = i % p0;
        A[(long)QCOL(p0 + c) * ld + r] = tzero<T>();
    }
    __syncthreads();
}

// Panel in shared memory as explicit V: zeros above the diagonal, 1 on it.
template <class T>
__device__ __forceinline__ void qr_explicit_v(T* P, int ldp, int pw) {
    for (int o = threadIdx.x; o < pw * pw; o += blockDim.x) {
        const int i = o / pw, r = o % pw;  // column i, row r
        if (r <= i) P[i * ldp + r] = (r == i) ? tone<T>() : tzero<T>();
    }
}

// Unblocked Householder factorisation of the panel P (R rows, zero-padded)
// with two barriers per column: thread 0 forms reflector j from alpha = P[j][j]
// and the squared norm below it (computed by the warp that updated the column
// in the previous step); then every warp applies H_j to its panel columns with
// the unscaled x (the scale 1/(alpha - beta) is applied inside the dot and the
// update), forms the next norm(s), and all threads scale the previous column,
// which no longer is read.  tau_j goes to Tm[j][j], beta_j to P[j][j].
// Pivoting (pmp != null, the panel's slice of the column map): before step j
// thread 0 picks the remaining column with the largest norm below row j-1
// (alpha^2 + ||x||^2), the columns are swapped in P and in pmp (a third
// barrier), and every warp keeps the norms of all its columns current.
template <class T>
__device__ void qr_panel(T* P, int ldp, int R, int pw, T* Tm, int nb, T* psc, double* red, int* pmp, double* nb2,
                         real_t<T>* met) {
    using RT = real_t<T>;
    __shared__ int ksh;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    const bool piv = pmp != nullptr;
    const int R4 = 4 * ceil_div(R, 4);
    if (!piv) {
        if (wid == 0) {
            const double t = col_norm2(P, 1, R);
            if (lane == 0) red[0] = t;
        }
    } else {
        for (int c = wid; c < pw; c += nw) {
            const double t = col_norm2(P + c * ldp, 1, R);
            if (lane == 0) {
                nb2[c] = t;
                met[c] = RT(dabs2(P[c * ldp]) + t);
            }
        }
    }
    __syncthreads();
    for (int j = 0; j < pw; ++j) {
        T* x = P + j * ldp;
        if (tid == 0) {
            int k = j;
            if (piv) {
                RT best = met[j];
                for (int c = j + 1; c < pw; ++c)
                    if (met[c] > best) {
                        best = met[c];
                        k = c;
                    }
                if (k != j) {
                    const int ti = pmp[j];
                    pmp[j] = pmp[k];
                    pmp[k] = ti;
                    const double tn = nb2[j];
                    nb2[j] = nb2[k];
                    nb2[k] = tn;
                }
                ksh = k;
            }
            T* xk = P + k * ldp;  // the column that becomes column j
            const double xn2 = piv ? nb2[j] : red[j & 1];
            const T alpha = xk[j];
            T tau = tzero<T>(), scale = tzero<T>();
            const double a2 = dabs2(alpha) + xn2;
            // a sub-column below (1e-30)^2 (float32) is treated as zero
            if (xn2 > 0.0 && a2 > (sizeof(RT) == 4 ? 1e-60 : 0.0)) {
                if constexpr (is_complex_v<T>) {
                    // beta = -sign(Re alpha) |(alpha, x)| (real), tau = (beta - alpha) / beta,
                    // scale = 1 / (alpha - beta), evaluated in float64
                    const double ar = alpha.x, ai = alpha.y;
                    const double beta = -copysign(sqrt(a2), ar);
                    tau = T{RT((beta - ar) / beta), RT(-ai / beta)};
                    const double zr = ar - beta, zi = ai, zz = zr * zr + zi * zi;
                    scale = T{RT(zr / zz), RT(-zi / zz)};
                    xk[j] = T{RT(beta), RT(0)};
                } else if (sizeof(T) == 4 && a2 >= 1e-36) {
                    const T beta = -tcopysign(tsqrt(T(a2)), alpha);
                    tau = (beta - alpha) / beta;
                    scale = T(1) / (alpha - beta);
                    xk[j] = beta;
                } else {  // float64 (and float32 columns too small for float32 arithmetic)
                    const double al = alpha;
                    const double beta = -copysign(sqrt(a2), al);
                    tau = T((beta - al) / beta);
                    scale = T(1.0 / (al - beta));
                    xk[j] = T(beta);
                }
            }
            Tm[j * nb + j] = tau;
            psc[j] = scale;
        }
        __syncthreads();
        if (piv) {
            const int k = ksh;
            if (k != j) {
                T* xk = P + k * ldp;
                for (int r = tid; r < R4; r += nt) {
                    const T t = x[r];
                    x[r] = xk[r];
                    xk[r] = t;
                }
            }
        }
        const T tau = Tm[j * nb + j], scale = psc[j];
        if (j > 0) {
            const T sp = psc[j - 1];
            T* xp = P + (j - 1) * ldp;
            for (int r = j + tid; r < R; r += nt) xp[r] *= sp;
        }
        if (piv) __syncthreads();
        for (int c = j + 1 + wid; c < pw; c += nw) {
            T* y = P + c * ldp;
            if (tau != tzero<T>()) {
                // x is scaled inside the dot: the product of two raw sub-columns
                // would underflow in float32 for entries below ~1e-19.
                // y <- H^H y = y - conj(tau) v (v^H y), v = (1, x scale)
                T s0 = tzero<T>(), s1 = tzero<T>();
                int r = j + 1 + lane;
                for (; r + 32 < R; r += 64) {
                    s0 += tconj_mul(x[r] * scale, y[r]);
                    s1 += tconj_mul(x[r + 32] * scale, y[r + 32]);
                }
                if (r < R) s0 += tconj_mul(x[r] * scale, y[r]);
                const T sdot = warp_sum(s0 + s1) + y[j];
                const T f = tconj(tau) * sdot, fs = f * scale;
                for (int rr = j + 1 + lane; rr < R; rr += 32) y[rr] -= fs * x[rr];
                __syncwarp();
                if (lane == 0) y[j] -= f;
            }
            if (piv) {
                __syncwarp();
                const double t = col_norm2(y, j + 2, R);
                if (lane == 0) {
                    nb2[c] = t;
                    met[c] = RT(dabs2(y[j + 1]) + t);
                }
            } else if (c == j + 1) {
                __syncwarp();
                const double t = col_norm2(y, j + 2, R);
                if (lane == 0) red[(j + 1) & 1] = t;
            }
        }
        __syncthreads();
    }
    {
        const int j = pw - 1;
        const T sp = psc[j];
        T* xp = P + j * ldp;
        for (int r = j + 1 + tid; r < R; r += nt) xp[r] *= sp;
    }
    __syncthreads();
}

// T of the compact WY form of the panel (explicit V in P, tau_j on Tm's
// diagonal): G = V^H V with the tiled product, then row i of T by one lane:
// T[i][j] = -tau_j sum_{l=i}^{j-1} T[i][l] G[l][j] for j > i (the columnwise
// recursion of Schreiber & Van Loan, read by rows), zeros below the diagonal.
template <class T, int NI>
__device__ void qr_t_matrix(const T* P, int ldp, int R, int pw, T* Tm, int nb, T* G, T* Wp) {
    for (int cb = 0; cb < pw; cb += QR_QG) {
        auto col = [&](int c) -> const T* { return cb + c < pw ? P + (cb + c) * ldp : nullptr; };
        qr_vty<T, NI>(P, ldp, pw, R, Wp, col, true);
        __syncthreads();
        const int nw = blockDim.x >> 5;
        for (int o = threadIdx.x; o < pw * QR_QG; o += blockDim.x) {
            const int i = o / QR_QG, c = o % QR_QG;
            if (cb + c < pw) {
                T s = tzero<T>();
                for (int w = 0; w < nw; ++w) s += Wp[w * 8 * NI * QR_QG + o];
                G[i * pw + cb + c] = s;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < pw) {
        const int i = threadIdx.x;
        for (int j = 0; j < i; ++j) Tm[i * nb + j] = tzero<T>();
        for (int j = i + 1; j < pw; ++j) {
            T s = tzero<T>();
            for (int l = i; l < j; ++l) s += Tm[i * nb + l] * G[l * pw + j];
            Tm[i * nb + j] = tzero<T>() - Tm[j * nb + j] * s;
        }
    }
    __syncthreads();
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

template <class T>
__global__ void __launch_bounds__(QR_THREADS) k_qr(QRJob<T> job) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = blockIdx.x;
    const int m = job.m, n = job.n, ld = job.ld, nb = job.nb;
    const int kk = min(m, n);
    const int ldp = qr_ldp<T>(m);
    T* A = job.A + (long)b * job.strideA;
    T* Tw = job.Tw + (long)b * job.strideT;
    const bool piv = job.pivot && job.mode == QR_R_ROWS;
    const int tid = threadIdx.x, nt = blockDim.x, nw = nt >> 5;
    const int lane = tid & 31, wid = tid >> 5;
    const int ni = qr_ni(nb);
    const int cap = 8 * ni;
    double* red = reinterpret_cast<double*>(smem_raw);
    T* P = reinterpret_cast<T*>(smem_raw + 64 * sizeof(double));
    T* Tm = P + (size_t)nb * ldp;
    T* G = Tm + nb * nb;
    T* Wp = G + nb * nb;
    T* W0 = Wp + (size_t)nw * cap * QR_QG;
    T* W1 = W0 + (size_t)cap * QR_QG;
    using RT = real_t<T>;
    double* nb2 = reinterpret_cast<double*>(W1 + (size_t)cap * QR_QG);
    RT* met = reinterpret_cast<RT*>(nb2 + nb);
    RT* cnrm = met + nb;
    int* pm = reinterpret_cast<int*>(cnrm + n);
    int* pm2 = pm + n;
    // the column map in shared memory: the given one, or the order pivoting chooses
    {
        const int* cin = job.colmap ? job.colmap + (long)b * n : nullptr;
        for (int c = tid; c < n; c += nt) pm[c] = (cin && !piv) ? cin[c] : c;
    }
    __syncthreads();
    const int* cm = pm;
    // 16-byte accesses to columns of A (rows p0 + r, r a multiple of 4)
    const bool vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (ld % 4 == 0);

    for (int p0 = 0; p0 < kk; p0 += nb) {
        const int pw = min(nb, kk - p0);
        const int R = m - p0;
        const int R4 = 4 * ceil_div(R, 4);
        if (piv) {
            // block pivoting: order the remaining columns by their norm below row
            // p0 (ties by position; non-finite norms last), so the panel takes the
            // largest ones
            for (int c = p0 + wid; c < n; c += nw) {
                const T* col = A + (long)pm[c] * ld + p0;
                RT s2 = RT(0);
                for (int r = lane; r < R; r += 32) s2 += tabs2(col[r]);
                s2 = warp_sum(s2);
                if (lane == 0) cnrm[c] = (s2 == s2) ? s2 : RT(-1);
            }
            __syncthreads();
            for (int c = p0 + tid; c < n; c += nt) {
                const RT v = cnrm[c];
                int rank = 0;
                for (int q = p0; q < n; ++q) {
                    const RT w = cnrm[q];
                    rank += (w > v) || (w == v && q < c);
                }
                pm2[p0 + rank] = pm[c];
            }
            __syncthreads();
            for (int c = p0 + tid; c < n; c += nt) pm[c] = pm2[c];
            __syncthreads();
        }
        for (int i = tid; i < pw * R4; i += nt) {
            const int c = i / R4, r = i % R4;
            P[c * ldp + r] = r < R ? A[(long)QCOL(p0 + c) * ld + p0 + r] : tzero<T>();
        }
        __syncthreads();
        qr_panel(P, ldp, R, pw, Tm, nb, W0, red, piv ? pm + p0 : nullptr, nb2, met);
        // write the factored panel (R above, reflectors below the diagonal) back
        for (int i = tid; i < pw * R; i += nt) {
            const int c = i / R, r = i % R;
            A[(long)QCOL(p0 + c) * ld + p0 + r] = P[c * ldp + r];
        }
        __syncthreads();
        qr_explicit_v(P, ldp, pw);
        __syncthreads();
        if (ni == 4) qr_t_matrix<T, 4>(P, ldp, R, pw, Tm, nb, G, Wp);
        else if (ni == 2) qr_t_matrix<T, 2>(P, ldp, R, pw, Tm, nb, G, Wp);
        else qr_t_matrix<T, 1>(P, ldp, R, pw, Tm, nb, G, Wp);
        // keep T for forming Q
        for (int i = tid; i < nb * nb; i += nt) Tw[(p0 / nb) * nb * nb + i] = Tm[i];
        // --- trailing update of columns p0+pw .. n-1
        if (p0 + pw < n)
            qr_block_apply_nb<T>(A, ld, m, p0, pw, p0 + pw, n, P, ldp, Tm, nb, Wp, W0, W1, true, cm, vec);
        __syncthreads();
    }

    // --- outputs
    T* out = job.out + (long)b * job.strideOut;
    if (job.mode == QR_R_ROWS) {
        for (int i = tid; i < n * n; i += nt) {
            const int r = i / n, c = i % n;
            out[i] = (r <= c && r < kk) ? A[(long)QCOL(c) * ld + r] : tzero<T>();
        }
        if (piv)
            for (int c = tid; c < n; c += nt) job.colmap[(long)b * n + c] = pm[c];
        return;
    }
    // QR_L_AND_Q / QR_L_ONLY: L = R^T (n x kk)
    for (int i = tid; i < n * kk; i += nt) {
        const int r = i / kk, c = i % kk;
        out[i] = (c <= r) ? A[(long)QCOL(r) * ld + c] : tzero<T>();
    }
    if (job.mode == QR_L_ONLY) return;
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
            P[c * ldp + r] = r < R ? A[(long)QCOL(p0 + c) * ld + p0 + r] : tzero<T>();
        }
        for (int i = tid; i < nb * nb; i += nt) Tm[i] = Tw[pi * nb * nb + i];
        __syncthreads();
        qr_explicit_v(P, ldp, pw);
        __syncthreads();
        if (p0 + pw < kk)
            qr_block_apply_nb<T>(A, ld, m, p0, pw, p0 + pw, kk, P, ldp, Tm, nb, Wp, W0, W1, false, cm, vec);
        qr_form_panel<T>(A, ld, m, p0, pw, P, ldp, Tm, nb, W0, W1, cm, vec);
    }
}

}  // namespace thc
