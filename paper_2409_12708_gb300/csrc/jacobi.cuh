// jacobi.cuh -- truncated SVD of one compression step (Fig. 3, SVD sweep).
//
// Input per term: Z (p x n, row-major) with Z^H Z = C^H C, where C is the site
// matrix [(chi_l, n_phys) x k] being truncated (Z = R from a block-pivoted
// Householder QR of C when C has at least as many rows as columns, Z = C
// otherwise).  One-sided Jacobi (Hestenes) rotates
// pairs of rows of Z until all rows are mutually orthogonal; rotations are
// unitary, so Z^H Z = C^H C is preserved and the rows end up as
// sigma_j v_j^H with v_j the right singular vectors of C (v_j^T for real C).  Rows are visited in
// a block ordering: blocks of R rows play a round-robin tournament, and one
// warp holds the 2R rows of a block pair in registers while it rotates their
// pairs, so shared-memory traffic is one read and write per R rotations of a
// row.
//
// Selection (float64, the truncation decision): sigma_j^2 = ||z_j||^2 is
// accumulated in double, rows are ranked by sigma, and the kept count follows
// the truncation rule (cap D_max; with tol > 0 the smallest k whose discarded
// weight is at most tol^2 of the total).
//
// Finalisation: with W the kept normalised rows (w_j = v_j^H), U = C W^H is
// normalised column by column and the carried matrix becomes
// M = N (I - F) W with F = W W^H - I (N = column norms of C W^H).  Then
// U M = C W^H (I - F) W, the orthogonal projector onto span(V_k) to second
// order in F, so the state is reproduced to rounding error even though the
// Jacobi rows are orthogonal only to the convergence threshold.  (Real rows:
// conjugation is the identity.)
#pragma once

#include <type_traits>

#include "common.cuh"
#include "scalar.cuh"

namespace thc {

template <class T>
struct JacobiJob {
    T* Z;              // p x n rows, modified in place (term b at Z + b*strideZ)
    long strideZ;
    int p, n;
    T* V;              // out: kout x n normalised kept rows (zero rows when dropped)
    long strideV;
    double* sv;        // out: kout singular values (0 for dropped rows)
    long strideSv;
    int* keep;         // out: kept count per term
    int kout;          // static output bond
    double tol;        // truncation tolerance (0 = cap only)
    double rot_tol;    // rotation threshold on |z_a.z_b| / (|z_a||z_b|)
    int max_sweeps;
    int* status;       // OR of DEV_* flags
    double* dbg;       // [8]: p, n and the rotations of the last sweep of the first
                       // matrix that did not converge (written once); [4..7] as
                       // counters: sweeps, matrices, sweeps and matrices with p >= 128
    int ps;            // rows of Z held in shared memory (the rest stay in global memory)
    const int* colmap; // optional per-term column permutation (n ints, stride n): Z's
                       // column c is column colmap[c] of C; V is written in C's order
};

// player at tournament position `pos` in round r (position 0 fixed)
__device__ __forceinline__ int rr_player(int pos, int r, int P2) {
    if (pos == 0) return 0;
    int q = pos - 1 + r;  // < 2 (P2 - 1) since pos, r < P2
    if (q >= P2 - 1) q -= P2 - 1;
    return q + 1;
}
// ---------------------------------------------------------------------------
// Row storage.  Rows [0, ps) of Z are copied to shared memory (Zs); rows
// [ps, p) stay in global memory (Zg, L2-resident).  Both are reached through
// generic pointers, so the sweep code is the same for either.
template <class T>
struct Rows {
    T* Zs;
    T* Zg;
    int ps, n;
    __device__ __forceinline__ T* operator()(int i) const { return i < ps ? Zs + (long)i * n : Zg + (long)i * n; }
};

// compile-time loop: f(std::integral_constant<int, I>{}) for I in [B, E)
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// Pair maps over the 2R rows one warp holds in registers: K = R disjoint pairs
// per step, all indices compile-time (the steps are unrolled).
template <int R, int S>
struct CrossShift {  // step S of the cross pairs: A_k with B_{(k+S) mod R}
    static constexpr int K = R;
    static constexpr int a(int k) { return k; }
    static constexpr int b(int k) { return R + (k + S) % R; }
};
// player at position pos of round r of the circle method over P2 players
__host__ __device__ constexpr int circle_player(int pos, int r, int P2) {
    return pos == 0 ? 0 : (pos - 1 + r) % (P2 - 1) + 1;
}
template <int R, int S>
struct CircleShift {  // round S of the circle method over the 2R rows
    static constexpr int K = R;
    static constexpr int a(int k) { return circle_player(k, S, 2 * R); }
    static constexpr int b(int k) { return circle_player(2 * R - 1 - k, S, 2 * R); }
};

// Launch shape per row length: R rows per block (at most 4, which keeps the
// unrolled steps small), so that the 2R rows of a block pair (NPL values per
// lane each) take at most 64 registers per lane,
// and 512 threads per CTA (256 where even R = 1 needs more registers).
template <class T, int NPL>
struct JacobiCfg {
    static constexpr int regs_per_row = NPL * (int)sizeof(T) / 4;
    static constexpr int raw = 32 / regs_per_row;
    static constexpr int R = raw >= 4 ? 4 : (raw >= 2 ? 2 : 1);
    static constexpr int threads = 2 * R * regs_per_row <= 64 ? 512 : 256;
};

// Row layout in registers: with VEC = 16 / sizeof(T), n a multiple of VEC and
// 16-byte aligned rows (`vec`), lane l holds the VEC-wide chunks starting at
// VEC*l + 32*VEC*q (16-byte accesses); otherwise columns l + 32*i.  Columns at
// or beyond n are held as zeros.
template <class T, int NPL>
__device__ __forceinline__ void load_row(T (&x)[NPL], const T* row, bool ok, int n, bool vec) {
    constexpr int VEC = 16 / (int)sizeof(T);
    const int lane = threadIdx.x & 31;
    if constexpr (NPL % VEC == 0) {
        if (vec) {
#pragma unroll
            for (int q = 0; q < NPL / VEC; ++q) {
                const int c = VEC * lane + 32 * VEC * q;
                if (ok && c < n) {
                    const uint4 u = *reinterpret_cast<const uint4*>(row + c);
                    const T* pu = reinterpret_cast<const T*>(&u);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) x[q * VEC + e] = pu[e];
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) x[q * VEC + e] = tzero<T>();
                }
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int c = lane + 32 * i;
        x[i] = (ok && c < n) ? row[c] : tzero<T>();
    }
}

template <class T, int NPL>
__device__ __forceinline__ void store_row(const T (&x)[NPL], T* row, int n, bool vec) {
    constexpr int VEC = 16 / (int)sizeof(T);
    const int lane = threadIdx.x & 31;
    if constexpr (NPL % VEC == 0) {
        if (vec) {
#pragma unroll
            for (int q = 0; q < NPL / VEC; ++q) {
                const int c = VEC * lane + 32 * VEC * q;
                if (c < n) {
                    uint4 u;
                    T* pu = reinterpret_cast<T*>(&u);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) pu[e] = x[q * VEC + e];
                    *reinterpret_cast<uint4*>(row + c) = u;
                }
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int c = lane + 32 * i;
        if (c < n) row[c] = x[i];
    }
}

// Reciprocal, quotient and reciprocal square root for the rotation
// parameters: the fast hardware approximations in float32 (arguments are kept
// in range by the power-of-two scaling of the matrix), the library functions
// in float64.
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }
__device__ __forceinline__ float fast_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double fast_rsqrt(double x) { return rsqrt(x); }

// Warp sums of NV per-lane values (NV a power of two, at most 32), every lane
// getting all NV totals: a reduce-scatter butterfly leaves value i's total on
// the 32/NV lanes of group i (lane / (32/NV)), and one shuffle per value
// broadcasts it from the group's first lane (NV - 1 + 5 - log2(NV) + NV
// shuffles instead of 5 NV for NV independent butterflies).
template <int NV, class RT>
__device__ __forceinline__ void warp_sums_all(RT (&v)[NV]) {
    static_assert(NV >= 1 && NV <= 32 && (NV & (NV - 1)) == 0, "power of two");
    const int lane = threadIdx.x & 31;
    RT w[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) w[i] = v[i];
#pragma unroll
    for (int lev = 0; (1 << lev) < NV; ++lev) {
        const int o = 16 >> lev;
        const int half = (NV >> lev) / 2;
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < NV / 2; ++i) {
            if (i < half) {
                const RT send = upper ? w[i] : w[half + i];
                const RT keep = upper ? w[half + i] : w[i];
                w[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
    }
    RT t = w[0];
#pragma unroll
    for (int o = 32 / NV / 2; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = __shfl_sync(0xffffffffu, t, i * (32 / NV));
}

// One step of K disjoint pair rotations on register-resident rows: every pair
// (X[a], X[b]) of the map PM with both rows valid (bits of `vrows`) and both
// norms above the floor is rotated so that the two rows become orthogonal.
//   * nrm holds the squared norms of the 2R rows (the same in every lane): they
//     are computed exactly when a visit loads its rows and then updated with
//     the rotation identities |a'|^2 = |a|^2 - t |a.b|, |b'|^2 = |b|^2 + t |a.b|.
//   * The K dot products a.b = sum a conj(b) are reduced by a reduce-scatter
//     butterfly: each level hands half of the remaining values to the partner
//     lane, so pair k's dot ends on the 32/K lanes with k = lane / (32/K).
//   * Those lanes decide and parametrise pair k's rotation in the storage
//     precision (float64 is scarce on this part); c, s, t |a.b| (and the phase
//     of a.b for complex rows) are broadcast from the first lane of each group.
// The rotation is the classical one-sided Jacobi rotation (Hestenes): with
// alpha = |a|^2, beta = |b|^2, gamma = a.b, zeta = (beta - alpha) / (2 gamma),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = c t:
// a' = c a - s b, b' = s a + c b.  Complex rows first take b to e b with
// e = gamma / |gamma|, which makes the dot real (|gamma|), so the same real
// rotation applies: a' = c a - s e b, b' = s conj(e) a + c b.  A pair is
// rotated when |gamma|^2 > rot_tol^2 alpha beta.  t may carry a few units of
// rounding; c gets one Newton step, so that c^2 + s^2 = 1 holds to rounding
// and the rotation stays unitary.
template <class T, int NPL, int NR, class PM>
__device__ __forceinline__ int rotate_regs(T (&X)[NR][NPL], real_t<T> (&nrm)[NR], unsigned vrows, real_t<T> rt2,
                                           real_t<T> floor2, unsigned& changed) {
    using RT = real_t<T>;
    constexpr bool CX = is_complex_v<T>;
    constexpr int K = PM::K;
    static_assert(K == 1 || K == 2 || K == 4 || K == 8, "pairs per step");
    const int lane = threadIdx.x & 31;
    T v[K];
    unsigned pvalid = 0;
    static_for<0, K>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr int a = PM::a(k), b = PM::b(k);
        T g = tzero<T>();
#pragma unroll
        for (int i = 0; i < NPL; ++i) g += tconj_mul(X[b][i], X[a][i]);
        v[k] = g;
        pvalid |= ((vrows >> a) & (vrows >> b) & 1u) << k;
    });
    // reduce-scatter over the pair index (compile-time indices: the kept half
    // moves to the front), then a full butterfly on the last value
#pragma unroll
    for (int lev = 0; (1 << lev) < K; ++lev) {
        const int o = 16 >> lev;
        const int half = (K >> lev) / 2;
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < K / 2; ++i) {
            if (i < half) {
                const T send = upper ? v[i] : v[half + i];
                const T keep = upper ? v[half + i] : v[i];
                v[i] = keep + shfl_xor(send, o);
            }
        }
    }
    T ga = v[0];
#pragma unroll
    for (int o = 32 / K / 2; o >= 1; o >>= 1) ga += shfl_xor(ga, o);
    const int my_pair = lane / (32 / K);
    RT al = RT(0), be = RT(0);
    static_for<0, K>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if (k == my_pair) {
            al = nrm[PM::a(k)];
            be = nrm[PM::b(k)];
        }
    });
    RT c = RT(1), s = RT(0), tg = RT(0);
    T ph = tone<T>();  // phase e of gamma (complex rows only)
    bool rot = false;
    const RT g2 = tabs2(ga);
    if (((pvalid >> my_pair) & 1u) && al > floor2 && be > floor2 && g2 > rt2 * (al * be)) {
        RT gr;  // the dot after the phase: gamma (real rows) or |gamma| (complex rows)
        if constexpr (CX) {
            const RT inv = fast_rsqrt(g2);
            gr = g2 * inv;
            ph = tscale(ga, inv);
        } else {
            gr = ga;
        }
        const RT zeta = fast_div(be - al, RT(2) * gr);
        const RT az = zeta < RT(0) ? -zeta : zeta;
        const RT q = RT(1) + zeta * zeta;
        const RT root = az < RT(1e18) ? q * fast_rsqrt(q) : az;
        const RT t = fast_div(tcopysign(RT(1), zeta), az + root);
        const RT u = RT(1) + t * t;
        RT cc = fast_rsqrt(u);
        cc = cc * (RT(1.5) - RT(0.5) * u * cc * cc);
        c = cc;
        s = cc * t;
        tg = t * gr;
        rot = true;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, rot);
    int nrot = 0;
    static_for<0, K>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr int a = PM::a(k), b = PM::b(k);
        constexpr int src = k * (32 / K);
        if ((bal >> src) & 1u) {
            const RT ck = __shfl_sync(0xffffffffu, c, src);
            const RT sk = __shfl_sync(0xffffffffu, s, src);
            const RT tgk = __shfl_sync(0xffffffffu, tg, src);
            if constexpr (CX) {
                const T e = shfl(ph, src);
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const T x = X[a][i], y = X[b][i];
                    X[a][i] = tscale(x, ck) - tscale(e * y, sk);
                    X[b][i] = tscale(tconj_mul(e, x), sk) + tscale(y, ck);
                }
            } else {
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const T x = X[a][i], y = X[b][i];
                    X[a][i] = ck * x - sk * y;
                    X[b][i] = sk * x + ck * y;
                }
            }
            nrm[a] -= tgk;
            nrm[b] += tgk;
            changed |= (1u << a) | (1u << b);
            ++nrot;
        }
    });
    return nrot;
}

// CTA-wide copy of `count` elements; 16-byte vector accesses when both ends
// are 16-byte aligned and the byte count is a multiple of 16.
template <class T>
__device__ __forceinline__ void cta_copy(T* dst, const T* src, long count) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0 &&
        (count * (long)sizeof(T)) % 16 == 0) {
        const long nv = count * (long)sizeof(T) / 16;
        uint4* d = reinterpret_cast<uint4*>(dst);
        const uint4* s = reinterpret_cast<const uint4*>(src);
        for (long i = tid; i < nv; i += nt) d[i] = s[i];
    } else {
        for (long i = tid; i < count; i += nt) dst[i] = src[i];
    }
}

// One sweep of the block ordering.  Rows are grouped in blocks of R; the
// blocks play a round-robin tournament, and a warp takes the 2R rows of a
// block pair (A, B) into registers once per visit, with their squared norms:
//   * in the first round (where every block plays once) it rotates all pairs
//     of A u B by the circle method (2R-1 steps of R pairs), which covers the
//     pairs inside A and inside B;
//   * in later rounds it rotates the R^2 cross pairs in R steps, step S pairing
//     A_k with B_{(k+S) mod R}.
// The steps are unrolled with compile-time pair maps (R <= 4 keeps the code
// within the instruction cache), so rows never move between registers.  Every
// pair of rows is rotated exactly once per sweep, as in the cyclic method,
// while each row is read and written once per R rotations instead of once per
// rotation.  Rows with ||z||^2 <= floor2 are numerically zero (below the
// rounding level of the matrix they came from) and are not rotated.
template <class T, int NPL, int R>
__device__ int jacobi_sweep_reg(const Rows<T>& rows, int p, int n, bool vec, real_t<T> rt2, real_t<T> floor2) {
    using RT = real_t<T>;
    static_assert(R >= 1 && R <= 4, "rows per block");
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nbk = ceil_div(p, R);
    const int P2 = nbk + (nbk & 1);
    constexpr unsigned lowR = (1u << R) - 1u;
    int myrot = 0;
    for (int rr = 0; rr < P2 - 1; ++rr) {
        for (int bp = wid; bp < P2 / 2; bp += nw) {
            const int A = rr_player(bp, rr, P2), Bk = rr_player(P2 - 1 - bp, rr, P2);
            T X[2 * R][NPL];
            RT nrm[2 * R];
            unsigned vrows = 0;
#pragma unroll
            for (int i = 0; i < 2 * R; ++i) {
                const int blk = i < R ? A : Bk;
                const int row = blk * R + (i < R ? i : i - R);
                const bool ok = blk < nbk && row < p;
                vrows |= (ok ? 1u : 0u) << i;
                load_row<T, NPL>(X[i], ok ? rows(row) : rows.Zs, ok, n, vec);
                RT s2 = RT(0);
#pragma unroll
                for (int e = 0; e < NPL; ++e) s2 += tabs2(X[i][e]);
                nrm[i] = s2;
            }
            warp_sums_all<2 * R>(nrm);
            unsigned changed = 0;
            if (rr == 0) {
                static_for<0, 2 * R - 1>([&](auto sc) {
                    myrot += rotate_regs<T, NPL, 2 * R, CircleShift<R, decltype(sc)::value>>(X, nrm, vrows, rt2,
                                                                                             floor2, changed);
                });
            } else if ((vrows & lowR) && (vrows >> R)) {
                static_for<0, R>([&](auto sc) {
                    myrot += rotate_regs<T, NPL, 2 * R, CrossShift<R, decltype(sc)::value>>(X, nrm, vrows, rt2,
                                                                                            floor2, changed);
                });
            }
            // rows no rotation touched are unchanged in memory
#pragma unroll
            for (int i = 0; i < 2 * R; ++i) {
                if ((vrows >> i) & (changed >> i) & 1u) {
                    const int blk = i < R ? A : Bk;
                    store_row<T, NPL>(X[i], rows(blk * R + (i < R ? i : i - R)), n, vec);
                }
            }
        }
        __syncthreads();
    }
    return myrot;
}

// Sweeps until a sweep applies no rotation (or the budget ends).
template <class T, int NPL>
__device__ int jacobi_rows(const Rows<T>& rows, int p, int n, bool vec, double rot_tol, double floor2,
                           int max_sweeps, int* nrot_sh, int* status, double* dbg) {
    constexpr int R = JacobiCfg<T, NPL>::R;
    const int lane = threadIdx.x & 31;
    if (p < 2) return 0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) *nrot_sh = 0;
        __syncthreads();
        const int myrot = jacobi_sweep_reg<T, NPL, R>(rows, p, n, vec, real_t<T>(rot_tol * rot_tol),
                                                      real_t<T>(floor2));
        if (lane == 0 && myrot) atomicAdd(nrot_sh, myrot);
        __syncthreads();
        const int total = *nrot_sh;
        __syncthreads();
        if (total == 0) return sweep + 1;
        if (sweep == max_sweeps - 1 && threadIdx.x == 0) {
            atomicOr(status, DEV_NONCONVERGED);
            if (dbg && atomicCAS(reinterpret_cast<unsigned long long*>(dbg), 0ull,
                                 (unsigned long long)__double_as_longlong((double)p)) == 0ull) {
                dbg[1] = n;
                dbg[2] = total;
            }
        }
    }
    return max_sweeps;
}

// One CTA (JacobiCfg threads) per term.  Dynamic smem: p doubles (sigma^2), p ints
// (order), then job.ps rows of Z.
template <class T, int NPL>
__global__ void __launch_bounds__(JacobiCfg<T, NPL>::threads) k_jacobi_select(JacobiJob<T> job) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int nrot_sh;
    __shared__ int kkeep_sh;
    constexpr int VEC = 16 / (int)sizeof(T);
    const int b = blockIdx.x;
    const int p = job.p, n = job.n, kout = job.kout;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    double* s2 = reinterpret_cast<double*>(smem_raw);
    int* order = reinterpret_cast<int*>(s2 + p);
    T* Zg = job.Z + (long)b * job.strideZ;
    T* Zs = reinterpret_cast<T*>(smem_raw + ((p * (sizeof(double) + sizeof(int)) + 15) & ~15));
    const int ps = min(job.ps, p);
    cta_copy(Zs, Zg, (long)ps * n);
    __syncthreads();
    const Rows<T> rows{Zs, Zg, ps, n};
    const bool vec = (n % VEC == 0) && ((reinterpret_cast<uintptr_t>(Zg) & 15) == 0);
    // A power-of-two scale (exact) taken from the largest entry brings the
    // matrix to max |z| in [0.5, 1), which keeps every square, norm and rotation
    // parameter clear of underflow and overflow whatever the input's magnitude.
    // The Frobenius norm (invariant under the rotations) of the scaled matrix
    // then sets the rounding floor.
    __shared__ double red[32];
    using RT = real_t<T>;
    RT tmax = RT(0);
    for (int r = wid; r < p; r += nw) {
        const T* z = rows(r);
        for (int c = lane; c < n; c += 32) tmax = fmax(tmax, tmaxabs(z[c]));
    }
    const double amax = block_max((double)tmax, red);
    double scale = 1.0;
    if (amax > 0.0 && amax < 1e300) {
        int ex = 0;
        frexp(amax, &ex);
        scale = ldexp(1.0, -ex);
    }
    RT tpart = RT(0);
    {
        const RT sc = RT(scale);
        for (int r = wid; r < p; r += nw) {
            T* z = rows(r);
            for (int c = lane; c < n; c += 32) {
                const T v = tscale(z[c], sc);
                z[c] = v;
                tpart += tabs2(v);
            }
        }
    }
    const double fro2 = block_sum((double)tpart, red);
    const double floor2 = Real<RT>::eps * Real<RT>::eps * fro2;
    const int sweeps = jacobi_rows<T, NPL>(rows, p, n, vec, job.rot_tol, floor2, job.max_sweeps, &nrot_sh,
                                           job.status, job.dbg);
    if (tid == 0 && job.dbg) {  // sweep statistics: all matrices, and those with p >= 128
        unsigned long long* st = reinterpret_cast<unsigned long long*>(job.dbg + 4);
        atomicAdd(st + 0, (unsigned long long)sweeps);
        atomicAdd(st + 1, 1ull);
        if (p >= 128) {
            atomicAdd(st + 2, (unsigned long long)sweeps);
            atomicAdd(st + 3, 1ull);
        }
    }
    __syncthreads();
    // squared row norms: per-lane partials in the storage precision, summed in
    // float64
    for (int r = wid; r < p; r += nw) {
        const T* z = rows(r);
        RT acc = RT(0);
        for (int c = lane; c < n; c += 32) acc += tabs2(z[c]);
        const double a = warp_sum((double)acc);
        if (lane == 0) s2[r] = a;
    }
    __syncthreads();
    // rank by descending sigma (ties by index): order[rank] = row.  The squared
    // norms are non-negative, so their bit patterns order like the values and
    // the comparisons run on the integer pipe.
    {
        const long long* s2i = reinterpret_cast<const long long*>(s2);
        for (int r = tid; r < p; r += nt) {
            const long long v = s2i[r];
            int rank = 0;
            for (int q = 0; q < p; ++q) {
                const long long w = s2i[q];
                rank += (w > v) || (w == v && q < r);
            }
            order[rank] = r;
        }
    }
    __syncthreads();
    if (tid == 0) {
        double total = 0.0;
        for (int q = 0; q < p; ++q) total += s2[q];
        int k = kout;
        if (job.tol > 0.0) {
            // smallest k with sum_{j>=k} sigma_j^2 <= tol^2 * total
            double tail = total;
            int kt = p;
            for (int q = 0; q < p; ++q) {
                if (tail <= job.tol * job.tol * total) { kt = q; break; }
                tail -= s2[order[q]];
            }
            if (kt == p && tail <= job.tol * job.tol * total) kt = p;
            k = max(1, min(kout, kt));
        }
        kkeep_sh = k;
        job.keep[b] = k;
        if (!(total == total) || total > 1e300) atomicOr(job.status, DEV_NONFINITE);
    }
    __syncthreads();
    const int k = kkeep_sh;
    // rows at or below twice the rounding floor are dropped (never rotated rows are
    // below the floor, so a kept row is always orthogonal to the threshold)
    const double thresh = 2.0 * Real<RT>::eps * sqrt(fro2);
    T* V = job.V + (long)b * job.strideV;
    double* sv = job.sv + (long)b * job.strideSv;
    for (int j = wid; j < kout; j += nw) {
        double sig = 0.0;
        int row = -1;
        if (j < k && j < p) {
            row = order[j];
            sig = sqrt(s2[row]);
            if (!(sig > thresh)) row = -1;
        }
        if (lane == 0) sv[j] = row >= 0 ? sig / scale : 0.0;
        const RT inv = row >= 0 ? RT(1.0 / sig) : RT(0);
        const T* z = row >= 0 ? rows(row) : nullptr;
        const int* cm = job.colmap ? job.colmap + (long)b * n : nullptr;
        for (int c = lane; c < n; c += 32) V[(long)j * n + (cm ? cm[c] : c)] = z ? tscale(z[c], inv) : tzero<T>();
    }
}

// Finalisation per term, step 1: normalise the columns of U (mU x kout,
// row-major, in place) and keep their norms nu (coalesced: thread j walks
// column j).  Steps 2 and 3 are batched GEMMs on the engine side:
// F = V V^T, then M = diag(nu) (I - F') V with F' = F - I on the kept rows.
template <class T>
__global__ void __launch_bounds__(256) k_unit_columns(T* U, long strideU, int mU, int kout, T* nu,
                                                      long strideNu) {
    const int b = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kout) return;
    U += (long)b * strideU;
    double acc = 0.0;
    for (int r = 0; r < mU; ++r) acc += (double)tabs2(U[(long)r * kout + j]);
    const double nrm = sqrt(acc);
    const real_t<T> inv = nrm > 0.0 ? real_t<T>(1.0 / nrm) : real_t<T>(0);
    for (int r = 0; r < mU; ++r) U[(long)r * kout + j] = tscale(U[(long)r * kout + j], inv);
    nu[(long)b * strideNu + j] = nrm > 0.0 ? treal<T>(real_t<T>(nrm)) : tzero<T>();
}

// A-operand of M = diag(nu) (I - F') V: element (i, l) = nu_i (delta_il - F'_il),
// F'_il = F_il - delta_il on kept (non-zero) rows, F' = 0 on dropped rows.
template <class T>
struct CorrA {
    const T* F;
    long sF;
    const T* nu;
    long sNu;
    int k;
    __device__ __forceinline__ T operator()(int b, int i, int l) const {
        const T f = F[(long)b * sF + (long)i * k + l];
        const T fii = F[(long)b * sF + (long)i * k + i];
        if (fii == tzero<T>()) return tzero<T>();  // dropped row: M row stays zero
        const T fp = (i == l) ? f - tone<T>() : f;
        return nu[(long)b * sNu + i] * ((i == l ? tone<T>() : tzero<T>()) - fp);
    }
};

}  // namespace thc
