// small.cuh -- single-CTA float64 kernels for the small dense problems:
//   * the eigen-decomposition t = U diag(lambda) U^T of App. D (kinetic term),
//   * the Krylov projected problems of Sec. 2.2: canonical orthogonalisation
//     of the overlap S, the effective matrix C^T Htil C (Eq. eff_H), its
//     eigen-decomposition, and the time-step coefficients exp(-i dt Heff) a(0).
// The eigensolver is the cyclic two-sided Jacobi method with the round-robin
// ordering (Golub & Van Loan, symmetric Schur decomposition), n <= 64; for the
// complex Hermitian problems of time evolution each rotation first takes the
// off-diagonal entry to a real one by a phase.
#pragma once

#include "common.cuh"
#include "scalar.cuh"

namespace thc {

constexpr int SMALL_MAX = 64;

// In shared memory: A (n x n, ld SMALL_MAX) symmetric, V (n x n) output
// eigenvectors (columns), cs scratch (2*SMALL_MAX doubles).  On return the
// eigenvalues sit on A's diagonal (unsorted).  All threads of the block call.
static __device__ void small_sym_eig(double* A, double* V, int n, double* cs, int* flag) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < n * n; i += nt) {
        const int r = i / n, c = i % n;
        V[r * SMALL_MAX + c] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (n < 2) return;
    const int P2 = n + (n & 1);
    __shared__ double offn;
    for (int sweep = 0; sweep < 60; ++sweep) {
        if (tid == 0) {
            double off = 0.0, tot = 0.0;
            for (int r = 0; r < n; ++r)
                for (int c = 0; c < n; ++c) {
                    const double x = A[r * SMALL_MAX + c] * A[r * SMALL_MAX + c];
                    tot += x;
                    if (r != c) off += x;
                }
            offn = (off <= 1e-30 * tot) ? -1.0 : off;
        }
        __syncthreads();
        if (offn < 0.0) return;
        for (int rnd = 0; rnd < P2 - 1; ++rnd) {
            // rotation parameters of the n/2 disjoint pairs of this round
            for (int pi = tid; pi < P2 / 2; pi += nt) {
                const int a = (pi == 0) ? 0 : ((pi - 1 + rnd) % (P2 - 1)) + 1;
                const int qpos = P2 - 1 - pi;
                const int bq = (qpos == 0) ? 0 : ((qpos - 1 + rnd) % (P2 - 1)) + 1;
                double c = 1.0, s = 0.0;
                const int p = min(a, bq), q = max(a, bq);
                if (q < n) {
                    const double apq = A[p * SMALL_MAX + q];
                    if (apq != 0.0) {
                        const double tau = (A[q * SMALL_MAX + q] - A[p * SMALL_MAX + p]) / (2.0 * apq);
                        const double t = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                cs[2 * pi] = c;
                cs[2 * pi + 1] = s;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int o = tid; o < (P2 / 2) * n; o += nt) {
                const int pi = o / n, j = o % n;
                const int a = (pi == 0) ? 0 : ((pi - 1 + rnd) % (P2 - 1)) + 1;
                const int qpos = P2 - 1 - pi;
                const int bq = (qpos == 0) ? 0 : ((qpos - 1 + rnd) % (P2 - 1)) + 1;
                const int p = min(a, bq), q = max(a, bq);
                if (q >= n) continue;
                const double c = cs[2 * pi], s = cs[2 * pi + 1];
                const double x = A[p * SMALL_MAX + j], y = A[q * SMALL_MAX + j];
                A[p * SMALL_MAX + j] = c * x - s * y;
                A[q * SMALL_MAX + j] = s * x + c * y;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int o = tid; o < (P2 / 2) * n; o += nt) {
                const int pi = o / n, i = o % n;
                const int a = (pi == 0) ? 0 : ((pi - 1 + rnd) % (P2 - 1)) + 1;
                const int qpos = P2 - 1 - pi;
                const int bq = (qpos == 0) ? 0 : ((qpos - 1 + rnd) % (P2 - 1)) + 1;
                const int p = min(a, bq), q = max(a, bq);
                if (q >= n) continue;
                const double c = cs[2 * pi], s = cs[2 * pi + 1];
                double x = A[i * SMALL_MAX + p], y = A[i * SMALL_MAX + q];
                A[i * SMALL_MAX + p] = c * x - s * y;
                A[i * SMALL_MAX + q] = s * x + c * y;
                x = V[i * SMALL_MAX + p];
                y = V[i * SMALL_MAX + q];
                V[i * SMALL_MAX + p] = c * x - s * y;
                V[i * SMALL_MAX + q] = s * x + c * y;
            }
            __syncthreads();
        }
    }
    if (tid == 0 && flag) atomicOr(flag, DEV_SMALL_NONCONV);
}

// ascending order of the diagonal of A (n entries) into ord
static __device__ void small_sort_diag(const double* A, int n, int* ord) {
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const double v = A[r * SMALL_MAX + r];
        int rank = 0;
        for (int q = 0; q < n; ++q) {
            const double w = A[q * SMALL_MAX + q];
            rank += (w < v) || (w == v && q < r);
        }
        ord[rank] = r;
    }
    __syncthreads();
}

// t (L x L row-major, device) -> lambda ascending, u (row-major, column i = eigvec i)
// dynamic shared memory: 2*SMALL_MAX^2 + 2*SMALL_MAX doubles + SMALL_MAX ints
constexpr size_t KINETIC_SMEM = (2 * SMALL_MAX * SMALL_MAX + 2 * SMALL_MAX) * sizeof(double) +
                                SMALL_MAX * sizeof(int);
static __global__ void k_kinetic_factors(int L, const double* t, double* lam, double* u, int* flag) {
    extern __shared__ __align__(16) double smd[];
    double* A = smd;
    double* V = A + SMALL_MAX * SMALL_MAX;
    double* cs = V + SMALL_MAX * SMALL_MAX;
    int* ord = reinterpret_cast<int*>(cs + 2 * SMALL_MAX);
    for (int i = threadIdx.x; i < L * L; i += blockDim.x) {
        const int r = i / L, c = i % L;
        A[r * SMALL_MAX + c] = 0.5 * (t[r * L + c] + t[c * L + r]);
    }
    __syncthreads();
    small_sym_eig(A, V, L, cs, flag);
    small_sort_diag(A, L, ord);
    for (int i = threadIdx.x; i < L; i += blockDim.x) lam[i] = A[ord[i] * SMALL_MAX + ord[i]];
    for (int i = threadIdx.x; i < L * L; i += blockDim.x) {
        const int r = i / L, c = i % L;
        u[r * L + c] = V[r * SMALL_MAX + ord[c]];
    }
}

constexpr size_t KRYLOV_SMEM = (3 * SMALL_MAX * SMALL_MAX + 6 * SMALL_MAX) * sizeof(double) +
                               2 * SMALL_MAX * sizeof(int);
// Krylov projected problem.  Ht, S: K x K device (row-major, float64).
// mode 0 (ground): ritz[K] ascending (NaN beyond the kept rank), coef_re[K] =
//   C y_0 (coefficients of the lowest Ritz vector on the v_i).
// mode 1 (time step): coef_re/coef_im[K] = C exp(-i dt Heff) C^T S e_0.
// info[0] = kept rank r, info[1] = flags.
static __global__ void k_krylov_small(int K, const double* Ht, const double* S, int mode, double dt,
                               double drop, double* ritz, double* coef_re, double* coef_im,
                               int* info) {
    extern __shared__ __align__(16) double smd[];
    double* A = smd;
    double* V = A + SMALL_MAX * SMALL_MAX;
    double* C = V + SMALL_MAX * SMALL_MAX;
    double* cs = C + SMALL_MAX * SMALL_MAX;
    double* w = cs + 2 * SMALL_MAX;
    double* b0 = w + SMALL_MAX;
    double* br = b0 + SMALL_MAX;
    double* bi = br + SMALL_MAX;
    int* ord = reinterpret_cast<int*>(bi + SMALL_MAX);
    int* keep = ord + SMALL_MAX;
    __shared__ int r_sh;
    __shared__ int flag;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) flag = 0;
    // canonical orthogonalisation: S = W s W^T, keep s > drop * max(s)
    for (int i = tid; i < K * K; i += nt) {
        const int r = i / K, c = i % K;
        A[r * SMALL_MAX + c] = 0.5 * (S[r * K + c] + S[c * K + r]);
    }
    __syncthreads();
    small_sym_eig(A, V, K, cs, &flag);
    if (tid == 0) {
        double smax = 0.0;
        for (int i = 0; i < K; ++i) smax = fmax(smax, A[i * SMALL_MAX + i]);
        int r = 0;
        for (int i = 0; i < K; ++i)
            if (A[i * SMALL_MAX + i] > drop * smax) keep[r++] = i;
        r_sh = r;
    }
    __syncthreads();
    const int r = r_sh;
    // C = W_keep s_keep^{-1/2}  (K x r)
    for (int i = tid; i < K * r; i += nt) {
        const int row = i / r, c = i % r;
        const int e = keep[c];
        C[row * SMALL_MAX + c] = V[row * SMALL_MAX + e] / sqrt(A[e * SMALL_MAX + e]);
    }
    __syncthreads();
    // Heff = C^T Htil_sym C  (r x r); reuse V as scratch for Htil_sym C (K x r)
    for (int i = tid; i < K * r; i += nt) {
        const int row = i / r, c = i % r;
        double s = 0.0;
        for (int l = 0; l < K; ++l)
            s += 0.5 * (Ht[row * K + l] + Ht[l * K + row]) * C[l * SMALL_MAX + c];
        V[row * SMALL_MAX + c] = s;
    }
    __syncthreads();
    for (int i = tid; i < r * r; i += nt) {
        const int a = i / r, c = i % r;
        double s = 0.0;
        for (int l = 0; l < K; ++l) s += C[l * SMALL_MAX + a] * V[l * SMALL_MAX + c];
        A[a * SMALL_MAX + c] = s;
    }
    __syncthreads();
    for (int i = tid; i < r * r; i += nt) {  // symmetrise
        const int a = i / r, c = i % r;
        if (a < c) {
            const double m = 0.5 * (A[a * SMALL_MAX + c] + A[c * SMALL_MAX + a]);
            A[a * SMALL_MAX + c] = m;
            A[c * SMALL_MAX + a] = m;
        }
    }
    __syncthreads();
    small_sym_eig(A, V, r, cs, &flag);
    small_sort_diag(A, r, ord);
    if (mode == 0) {
        for (int i = tid; i < K; i += nt) ritz[i] = i < r ? A[ord[i] * SMALL_MAX + ord[i]] : nan("");
        for (int i = tid; i < K; i += nt) {
            double s = 0.0;
            for (int c = 0; c < r; ++c) s += C[i * SMALL_MAX + c] * V[c * SMALL_MAX + ord[0]];
            coef_re[i] = s;
        }
    } else {
        // b0 = C^T S e_0 (coordinates of v_0 in the orthonormalised basis)
        for (int c = tid; c < r; c += nt) {
            double s = 0.0;
            for (int l = 0; l < K; ++l) s += C[l * SMALL_MAX + c] * 0.5 * (S[l * K + 0] + S[0 * K + l]);
            b0[c] = s;
        }
        __syncthreads();
        // w = Y^T b0, then phase, then b = Y w
        for (int j = tid; j < r; j += nt) {
            double s = 0.0;
            for (int c = 0; c < r; ++c) s += V[c * SMALL_MAX + j] * b0[c];
            w[j] = s;
        }
        __syncthreads();
        for (int c = tid; c < r; c += nt) {
            double sr = 0.0, si = 0.0;
            for (int j = 0; j < r; ++j) {
                const double e = A[j * SMALL_MAX + j];
                double sn, cn;
                sincos(-dt * e, &sn, &cn);
                sr += V[c * SMALL_MAX + j] * cn * w[j];
                si += V[c * SMALL_MAX + j] * sn * w[j];
            }
            br[c] = sr;
            bi[c] = si;
        }
        __syncthreads();
        for (int i = tid; i < K; i += nt) {
            double sr = 0.0, si = 0.0;
            for (int c = 0; c < r; ++c) {
                sr += C[i * SMALL_MAX + c] * br[c];
                si += C[i * SMALL_MAX + c] * bi[c];
            }
            coef_re[i] = sr;
            coef_im[i] = si;
        }
    }
    __syncthreads();
    if (tid == 0) {
        info[0] = r;
        info[1] = flag;
    }
}

// ---------------------------------------------------------------------------
// Complex Hermitian counterparts (complex Krylov vectors of a time evolution).

// Hermitian Jacobi on A (n x n, ld SMALL_MAX, shared memory); V receives the
// unitary eigenvector matrix (columns), the real eigenvalues end on A's
// diagonal (unsorted).  Rotation of the pair (p, q) with a_pq = |a_pq| e^{i th}:
// U = diag(1, e^{-i th}) J, J the real Jacobi rotation of the phased block
// [[a_pp, |a_pq|], [|a_pq|, a_qq]]; A <- U^H A U, V <- V U.  cs: 2*SMALL_MAX
// doubles, ph: SMALL_MAX phases.  All threads of the block call.
static __device__ void small_herm_eig(c64* A, c64* V, int n, double* cs, c64* ph, int* flag) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < n * n; i += nt) {
        const int r = i / n, c = i % n;
        V[r * SMALL_MAX + c] = (r == c) ? c64{1.0, 0.0} : c64{0.0, 0.0};
    }
    __syncthreads();
    if (n < 2) return;
    const int P2 = n + (n & 1);
    __shared__ double offn;
    for (int sweep = 0; sweep < 60; ++sweep) {
        if (tid == 0) {
            double off = 0.0, tot = 0.0;
            for (int r = 0; r < n; ++r)
                for (int c = 0; c < n; ++c) {
                    const double x = tabs2(A[r * SMALL_MAX + c]);
                    tot += x;
                    if (r != c) off += x;
                }
            offn = (off <= 1e-30 * tot) ? -1.0 : off;
        }
        __syncthreads();
        if (offn < 0.0) return;
        for (int rnd = 0; rnd < P2 - 1; ++rnd) {
            for (int pi = tid; pi < P2 / 2; pi += nt) {
                const int a = (pi == 0) ? 0 : ((pi - 1 + rnd) % (P2 - 1)) + 1;
                const int qpos = P2 - 1 - pi;
                const int bq = (qpos == 0) ? 0 : ((qpos - 1 + rnd) % (P2 - 1)) + 1;
                double c = 1.0, s = 0.0;
                c64 e{1.0, 0.0};
                const int p = min(a, bq), q = max(a, bq);
                if (q < n) {
                    const c64 apq = A[p * SMALL_MAX + q];
                    const double g = sqrt(tabs2(apq));
                    if (g != 0.0) {
                        e = c64{apq.x / g, apq.y / g};
                        const double tau = (A[q * SMALL_MAX + q].x - A[p * SMALL_MAX + p].x) / (2.0 * g);
                        const double t = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                cs[2 * pi] = c;
                cs[2 * pi + 1] = s;
                ph[pi] = e;
            }
            __syncthreads();
            // rows: A <- U^H A  (row_p <- c row_p - s e row_q, row_q <- s row_p + c e row_q)
            for (int o = tid; o < (P2 / 2) * n; o += nt) {
                const int pi = o / n, j = o % n;
                const int a = (pi == 0) ? 0 : ((pi - 1 + rnd) % (P2 - 1)) + 1;
                const int qpos = P2 - 1 - pi;
                const int bq = (qpos == 0) ? 0 : ((qpos - 1 + rnd) % (P2 - 1)) + 1;
                const int p = min(a, bq), q = max(a, bq);
                if (q >= n) continue;
                const double c = cs[2 * pi], s = cs[2 * pi + 1];
                const c64 e = ph[pi];
                const c64 x = A[p * SMALL_MAX + j], y = A[q * SMALL_MAX + j];
                A[p * SMALL_MAX + j] = c * x - s * (e * y);
                A[q * SMALL_MAX + j] = s * x + c * (e * y);
            }
            __syncthreads();
            // columns: A <- A U, V <- V U  (col_p <- c col_p - s conj(e) col_q,
            // col_q <- s col_p + c conj(e) col_q)
            for (int o = tid; o < (P2 / 2) * n; o += nt) {
                const int pi = o / n, i = o % n;
                const int a = (pi == 0) ? 0 : ((pi - 1 + rnd) % (P2 - 1)) + 1;
                const int qpos = P2 - 1 - pi;
                const int bq = (qpos == 0) ? 0 : ((qpos - 1 + rnd) % (P2 - 1)) + 1;
                const int p = min(a, bq), q = max(a, bq);
                if (q >= n) continue;
                const double c = cs[2 * pi], s = cs[2 * pi + 1];
                const c64 ec = tconj(ph[pi]);
                c64 x = A[i * SMALL_MAX + p], y = A[i * SMALL_MAX + q];
                A[i * SMALL_MAX + p] = c * x - s * (ec * y);
                A[i * SMALL_MAX + q] = s * x + c * (ec * y);
                x = V[i * SMALL_MAX + p];
                y = V[i * SMALL_MAX + q];
                V[i * SMALL_MAX + p] = c * x - s * (ec * y);
                V[i * SMALL_MAX + q] = s * x + c * (ec * y);
            }
            __syncthreads();
        }
    }
    if (tid == 0 && flag) atomicOr(flag, DEV_SMALL_NONCONV);
}

// ascending order of the (real) diagonal of a complex Hermitian A into ord
static __device__ void small_sort_diag_c(const c64* A, int n, int* ord) {
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const double v = A[r * SMALL_MAX + r].x;
        int rank = 0;
        for (int q = 0; q < n; ++q) {
            const double w = A[q * SMALL_MAX + q].x;
            rank += (w < v) || (w == v && q < r);
        }
        ord[rank] = r;
    }
    __syncthreads();
}

constexpr size_t KRYLOV_SMEM_C = 3 * SMALL_MAX * SMALL_MAX * sizeof(c64) + 2 * SMALL_MAX * sizeof(double) +
                                 4 * SMALL_MAX * sizeof(c64) + SMALL_MAX * sizeof(double) +
                                 2 * SMALL_MAX * sizeof(int);
// Complex Krylov projected problem (Sec. 2.2, Eq. reortho / Eq. eff_H): the
// same steps as k_krylov_small with Hermitian Htil and S (K x K row-major c64).
// mode 0: ritz[K] ascending (NaN beyond the kept rank), coef[K] = C y_0.
// mode 1: coef[K] = C exp(-i dt Heff) C^H S e_0.  info[0] = kept rank.
static __global__ void k_krylov_small_c(int K, const c64* Ht, const c64* S, int mode, double dt, double drop,
                                 double* ritz, c64* coef, int* info) {
    extern __shared__ __align__(16) unsigned char smc[];
    c64* A = reinterpret_cast<c64*>(smc);
    c64* V = A + SMALL_MAX * SMALL_MAX;
    c64* C = V + SMALL_MAX * SMALL_MAX;
    double* cs = reinterpret_cast<double*>(C + SMALL_MAX * SMALL_MAX);
    c64* ph = reinterpret_cast<c64*>(cs + 2 * SMALL_MAX);
    c64* w = ph + SMALL_MAX;
    c64* b0 = w + SMALL_MAX;
    c64* bb = b0 + SMALL_MAX;
    double* sdiag = reinterpret_cast<double*>(bb + SMALL_MAX);
    int* ord = reinterpret_cast<int*>(sdiag + SMALL_MAX);
    int* keep = ord + SMALL_MAX;
    __shared__ int r_sh;
    __shared__ int flag;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) flag = 0;
    // canonical orthogonalisation: S = W s W^H, keep s > drop * max(s)
    for (int i = tid; i < K * K; i += nt) {
        const int r = i / K, c = i % K;
        A[r * SMALL_MAX + c] = 0.5 * (S[r * K + c] + tconj(S[c * K + r]));
    }
    __syncthreads();
    small_herm_eig(A, V, K, cs, ph, &flag);
    for (int i = tid; i < K; i += nt) sdiag[i] = A[i * SMALL_MAX + i].x;
    __syncthreads();
    if (tid == 0) {
        double smax = 0.0;
        for (int i = 0; i < K; ++i) smax = fmax(smax, sdiag[i]);
        int r = 0;
        for (int i = 0; i < K; ++i)
            if (sdiag[i] > drop * smax) keep[r++] = i;
        r_sh = r;
    }
    __syncthreads();
    const int r = r_sh;
    // C = W_keep s_keep^{-1/2}  (K x r)
    for (int i = tid; i < K * r; i += nt) {
        const int row = i / r, c = i % r;
        const int e = keep[c];
        C[row * SMALL_MAX + c] = V[row * SMALL_MAX + e] * (1.0 / sqrt(sdiag[e]));
    }
    __syncthreads();
    // Heff = C^H Htil_h C with Htil_h = (Htil + Htil^H) / 2; V holds Htil_h C
    for (int i = tid; i < K * r; i += nt) {
        const int row = i / r, c = i % r;
        c64 s{0.0, 0.0};
        for (int l = 0; l < K; ++l)
            s += (0.5 * (Ht[row * K + l] + tconj(Ht[l * K + row]))) * C[l * SMALL_MAX + c];
        V[row * SMALL_MAX + c] = s;
    }
    __syncthreads();
    for (int i = tid; i < r * r; i += nt) {
        const int a = i / r, c = i % r;
        c64 s{0.0, 0.0};
        for (int l = 0; l < K; ++l) s += tconj_mul(C[l * SMALL_MAX + a], V[l * SMALL_MAX + c]);
        A[a * SMALL_MAX + c] = s;
    }
    __syncthreads();
    for (int i = tid; i < r * r; i += nt) {  // Hermitian part
        const int a = i / r, c = i % r;
        if (a < c) {
            const c64 m = 0.5 * (A[a * SMALL_MAX + c] + tconj(A[c * SMALL_MAX + a]));
            A[a * SMALL_MAX + c] = m;
            A[c * SMALL_MAX + a] = tconj(m);
        } else if (a == c) {
            A[a * SMALL_MAX + a].y = 0.0;
        }
    }
    __syncthreads();
    small_herm_eig(A, V, r, cs, ph, &flag);
    small_sort_diag_c(A, r, ord);
    if (mode == 0) {
        for (int i = tid; i < K; i += nt) ritz[i] = i < r ? A[ord[i] * SMALL_MAX + ord[i]].x : nan("");
        for (int i = tid; i < K; i += nt) {
            c64 s{0.0, 0.0};
            for (int c = 0; c < r; ++c) s += C[i * SMALL_MAX + c] * V[c * SMALL_MAX + ord[0]];
            coef[i] = s;
        }
    } else {
        // b0 = C^H S_h e_0 (coordinates of v_0 in the orthonormalised basis)
        for (int c = tid; c < r; c += nt) {
            c64 s{0.0, 0.0};
            for (int l = 0; l < K; ++l)
                s += tconj_mul(C[l * SMALL_MAX + c], 0.5 * (S[l * K + 0] + tconj(S[0 * K + l])));
            b0[c] = s;
        }
        __syncthreads();
        // w = Y^H b0, phases exp(-i dt e_j), then bb = Y w
        for (int j = tid; j < r; j += nt) {
            c64 s{0.0, 0.0};
            for (int c = 0; c < r; ++c) s += tconj_mul(V[c * SMALL_MAX + j], b0[c]);
            double sn, cn;
            sincos(-dt * A[j * SMALL_MAX + j].x, &sn, &cn);
            w[j] = c64{cn, sn} * s;
        }
        __syncthreads();
        for (int c = tid; c < r; c += nt) {
            c64 s{0.0, 0.0};
            for (int j = 0; j < r; ++j) s += V[c * SMALL_MAX + j] * w[j];
            bb[c] = s;
        }
        __syncthreads();
        for (int i = tid; i < K; i += nt) {
            c64 s{0.0, 0.0};
            for (int c = 0; c < r; ++c) s += C[i * SMALL_MAX + c] * bb[c];
            coef[i] = s;
        }
    }
    __syncthreads();
    if (tid == 0) {
        info[0] = r;
        info[1] = flag;
    }
}

}  // namespace thc
