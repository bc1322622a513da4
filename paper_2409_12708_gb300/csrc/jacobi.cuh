// jacobi.cuh -- truncated SVD of one compression step (Fig. 3, SVD sweep).
//
// Input per term: Z (p x n, row-major) with Z^T Z = C^T C, where C is the site
// matrix [(chi_l, n_phys) x k] being truncated (Z = R from a Householder QR of
// C when C is tall, Z = C otherwise).  One-sided Jacobi (Hestenes) rotates
// pairs of rows of Z until all rows are mutually orthogonal; rotations are
// orthogonal, so Z^T Z = C^T C is preserved and the rows end up as
// sigma_j v_j^T with v_j the right singular vectors of C.  Rows are paired by
// the round-robin (tournament) ordering, p/2 disjoint pairs per round, one warp
// per pair with the two rows held in registers.
//
// Selection (float64, the truncation decision): sigma_j^2 = ||z_j||^2 is
// accumulated in double, rows are ranked by sigma, and the kept count follows
// the truncation rule (cap D_max; with tol > 0 the smallest k whose discarded
// weight is at most tol^2 of the total).
//
// Finalisation: with V_k the kept normalised rows, U = C V_k is normalised
// column by column and the carried matrix becomes M = N (I - F) V_k^T with
// F = V_k^T V_k - I (N = column norms of C V_k).  Then U M = C V_k (I-F) V_k^T,
// the orthogonal projector onto span(V_k) to second order in F, so the state
// is reproduced to rounding error even though the Jacobi rows are orthogonal
// only to the convergence threshold.
#pragma once

#include "common.cuh"

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
    double* dbg;       // [8]: p, n, rotations and max cosine of the last sweep of the
                       // first matrix that did not converge (written once); [4..7] as
                       // counters: sweeps, matrices, sweeps and matrices with p >= 128
    int blk;           // row block of the blocked ordering (slot of 2*blk rows)
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

// Rotate up to K (1, 2 or 4) independent pairs of rows at once (rows ra[i],
// rb[i], for the i set in the bit mask `valid`) so that every pair becomes
// orthogonal.  The K pairs are
// interleaved so their loads, reductions and scalar chains overlap.
//   * Row layout per lane: with VEC = 16 / sizeof(T) and n a multiple of VEC
//     (and 16-byte aligned rows), lane l owns the VEC-wide chunks starting at
//     VEC*l + 32*VEC*q and moves them with 16-byte accesses; otherwise lane l
//     owns columns l + 32*i.
//   * The 3K sums (|a|^2, |b|^2, a.b per pair) are reduced by a reduce-scatter
//     butterfly: each level hands half of the remaining values to the partner
//     lane, so pair k's three sums end on the 32/K lanes with k = lane / (32/K).
//   * Those lanes decide and parametrise pair k's rotation in the storage
//     precision (float64 is scarce on this part) and the parameters are
//     broadcast from the first lane of each group.
template <class T, int NPL, int K>
__device__ __forceinline__ int rotate_pairs(T* const (&ra)[K], T* const (&rb)[K], unsigned valid, int n,
                                            T rot_tol, T floor2, T& mycos) {
    static_assert(K == 1 || K == 2 || K == 4, "pairs in flight");
    constexpr int VEC = 16 / (int)sizeof(T);
    const int lane = threadIdx.x & 31;
    const bool vec = (NPL % VEC == 0) && (n % VEC == 0);
    T xa[K][NPL], xb[K][NPL];
    // ---- loads
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (vec) {
#pragma unroll
            for (int q = 0; q < NPL / VEC; ++q) {
                const int c = VEC * lane + 32 * VEC * q;
                if (((valid >> k) & 1u) && c < n) {
                    const uint4 va = *reinterpret_cast<const uint4*>(ra[k] + c);
                    const uint4 vb = *reinterpret_cast<const uint4*>(rb[k] + c);
                    const T* pa = reinterpret_cast<const T*>(&va);
                    const T* pb = reinterpret_cast<const T*>(&vb);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        xa[k][q * VEC + e] = pa[e];
                        xb[k][q * VEC + e] = pb[e];
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) xa[k][q * VEC + e] = xb[k][q * VEC + e] = T(0);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                const int c = lane + 32 * i;
                const bool ok = ((valid >> k) & 1u) && c < n;
                xa[k][i] = ok ? ra[k][c] : T(0);
                xb[k][i] = ok ? rb[k][c] : T(0);
            }
        }
    }
    // ---- partial sums, value index v = 3k + {0: |a|^2, 1: |b|^2, 2: a.b}
    T v[3 * K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            s0 += xa[k][i] * xa[k][i];
            s1 += xb[k][i] * xb[k][i];
            s2 += xa[k][i] * xb[k][i];
        }
        v[3 * k] = s0;
        v[3 * k + 1] = s1;
        v[3 * k + 2] = s2;
    }
    // ---- reduce-scatter over the pair index (all indices compile-time: the kept
    // half moves to the front), then full butterflies on the last 3 values
#pragma unroll
    for (int lev = 0; (1 << lev) < K; ++lev) {
        const int o = 16 >> lev;
        const int half = (3 * K >> lev) / 2;
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < 3 * K / 2; ++i) {
            if (i < half) {
                const T send = upper ? v[i] : v[half + i];
                const T keep = upper ? v[half + i] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
    }
    // this lane carries (|a|^2, |b|^2, a.b) of pair k = lane / (32/K)
    T al = v[0], be = v[1], ga = v[2];
#pragma unroll
    for (int o = 32 / K / 2; o >= 1; o >>= 1) {
        al += __shfl_xor_sync(0xffffffffu, al, o);
        be += __shfl_xor_sync(0xffffffffu, be, o);
        ga += __shfl_xor_sync(0xffffffffu, ga, o);
    }
    const int my_pair = lane / (32 / K);
    T c = T(1), s = T(0);
    bool rot = false;
    if (((valid >> my_pair) & 1u) && al > floor2 && be > floor2) {
        const T nab = tsqrt(al) * tsqrt(be);
        const T ag = ga < T(0) ? -ga : ga;
        const T cosv = ag / nab;
        mycos = mycos > cosv ? mycos : cosv;
        if (ag > rot_tol * nab) {
            const T zeta = (be - al) / (T(2) * ga);
            const T az = zeta < T(0) ? -zeta : zeta;
            const T t = tcopysign(T(1), zeta) / (az + tsqrt(T(1) + zeta * zeta));
            c = T(1) / tsqrt(T(1) + t * t);
            s = c * t;
            rot = true;
        }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, rot);
    int nrot = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int src = k * (32 / K);
        if (!((bal >> src) & 1u)) continue;
        const T ck = __shfl_sync(0xffffffffu, c, src);
        const T sk = __shfl_sync(0xffffffffu, s, src);
        if (vec) {
#pragma unroll
            for (int q = 0; q < NPL / VEC; ++q) {
                const int col = VEC * lane + 32 * VEC * q;
                if (col < n) {
                    uint4 va, vb;
                    T* pa = reinterpret_cast<T*>(&va);
                    T* pb = reinterpret_cast<T*>(&vb);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        const T x = xa[k][q * VEC + e], y = xb[k][q * VEC + e];
                        pa[e] = ck * x - sk * y;
                        pb[e] = sk * x + ck * y;
                    }
                    *reinterpret_cast<uint4*>(ra[k] + col) = va;
                    *reinterpret_cast<uint4*>(rb[k] + col) = vb;
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                const int col = lane + 32 * i;
                if (col < n) {
                    ra[k][col] = ck * xa[k][i] - sk * xb[k][i];
                    rb[k][col] = sk * xa[k][i] + ck * xb[k][i];
                }
            }
        }
        ++nrot;
    }
    return nrot;
}

// pairs per warp in flight: as many as keep the two rows of every pair within
// 64 registers per lane (4 at most)
template <class T, int NPL>
struct PairsInFlight {
    static constexpr int raw = 128 / (NPL * (int)sizeof(T));
    static constexpr int value = raw >= 4 ? 4 : (raw >= 2 ? 2 : 1);
};

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

// Rows with ||z||^2 <= floor2 are numerically zero (below the rounding level of
// the matrix they came from): they are not rotated, and the selection drops them.
//
// Round-robin ordering over all p rows held in shared memory: p/2 disjoint
// pairs per round, JK of them per warp at a time.
template <class T, int NPL>
__device__ int jacobi_sweep_smem(T* Z, int p, int n, int r0_unused, T rot_tol, T floor2, T& mycos) {
    constexpr int JK = PairsInFlight<T, NPL>::value;
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int P2 = p + (p & 1);
    int myrot = 0;
    for (int r = 0; r < P2 - 1; ++r) {
        for (int pi0 = wid * JK; pi0 < P2 / 2; pi0 += nw * JK) {
            T* ra[JK];
            T* rb[JK];
            unsigned valid = 0;
#pragma unroll
            for (int k = 0; k < JK; ++k) {
                const int pi = pi0 + k;
                int a = p, b = p;
                if (pi < P2 / 2) {
                    a = rr_player(pi, r, P2);
                    b = rr_player(P2 - 1 - pi, r, P2);
                }
                const bool ok = a < p && b < p;
                ra[k] = ok ? Z + (long)a * n : Z;
                rb[k] = ok ? Z + (long)b * n : Z;
                valid |= (ok ? 1u : 0u) << k;
            }
            myrot += rotate_pairs<T, NPL, JK>(ra, rb, valid, n, rot_tol, floor2, mycos);
        }
        __syncthreads();
    }
    return myrot;
}

// Blocked ordering for Z too large for shared memory (Z stays in global
// memory, L2-resident).  Rows are grouped in blocks of bs.  A sweep first
// orthogonalises every block internally (round-robin inside the block), then
// visits every pair of blocks once (round-robin over blocks); for a visited
// pair (A, B) the CTA copies both blocks to shared memory and rotates the bs^2
// cross pairs in bs shift rounds, round s pairing A_i with B_{(i+s) mod bs}:
// bs independent pairs per round, JK per warp.  Every pair of rows is rotated
// exactly once per sweep, as in the cyclic method.
template <class T, int NPL>
__device__ int jacobi_sweep_blocked(T* Z, int p, int n, int bs, T* slot, T rot_tol, T floor2, T& mycos) {
    constexpr int JK = PairsInFlight<T, NPL>::value;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int wid = tid >> 5, nw = nt >> 5;
    const int nbk = ceil_div(p, bs);
    const int P2 = nbk + (nbk & 1);
    int myrot = 0;
    // intra-block pairs
    for (int kb = 0; kb < nbk; ++kb) {
        const int r0 = kb * bs, nr = min(bs, p - r0);
        cta_copy(slot, Z + (long)r0 * n, (long)nr * n);
        __syncthreads();
        myrot += jacobi_sweep_smem<T, NPL>(slot, nr, n, 0, rot_tol, floor2, mycos);
        cta_copy(Z + (long)r0 * n, slot, (long)nr * n);
        __syncthreads();
    }
    // cross-block pairs
    for (int rr = 0; rr < P2 - 1; ++rr) {
        for (int bp = 0; bp < P2 / 2; ++bp) {
            const int A = rr_player(bp, rr, P2), Bk = rr_player(P2 - 1 - bp, rr, P2);
            if (A >= nbk || Bk >= nbk) continue;
            const int ra0 = A * bs, na = min(bs, p - ra0);
            const int rb0 = Bk * bs, nb = min(bs, p - rb0);
            T* sa = slot;
            T* sb = slot + (size_t)bs * n;
            cta_copy(sa, Z + (long)ra0 * n, (long)na * n);
            cta_copy(sb, Z + (long)rb0 * n, (long)nb * n);
            __syncthreads();
            for (int sh = 0; sh < bs; ++sh) {
                for (int i0 = wid * JK; i0 < bs; i0 += nw * JK) {
                    T* ra[JK];
                    T* rb[JK];
                    unsigned valid = 0;
#pragma unroll
                    for (int k = 0; k < JK; ++k) {
                        const int i = i0 + k;
                        int j = i + sh;  // (i + sh) mod bs, both < bs
                        if (j >= bs) j -= bs;
                        const bool ok = i < na && j < nb;
                        ra[k] = ok ? sa + (long)i * n : slot;
                        rb[k] = ok ? sb + (long)j * n : slot;
                        valid |= (ok ? 1u : 0u) << k;
                    }
                    myrot += rotate_pairs<T, NPL, JK>(ra, rb, valid, n, rot_tol, floor2, mycos);
                }
                __syncthreads();
            }
            cta_copy(Z + (long)ra0 * n, sa, (long)na * n);
            cta_copy(Z + (long)rb0 * n, sb, (long)nb * n);
            __syncthreads();
        }
    }
    return myrot;
}

// Sweeps until a sweep applies no rotation (or the budget ends).  mode 1: Z in
// shared memory; mode 0: Z in global memory with the blocked ordering.
template <class T, int NPL>
__device__ int jacobi_rows(T* Z, int p, int n, int in_smem, int bs, T* slot, double rot_tol, double floor2,
                           int max_sweeps, int* nrot_sh, unsigned long long* maxcos_sh, int* status,
                           double* dbg) {
    const int lane = threadIdx.x & 31;
    if (p < 2) return 0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) {
            *nrot_sh = 0;
            *maxcos_sh = 0ull;
        }
        __syncthreads();
        T mycos = T(0);
        const T rt = T(rot_tol), f2 = T(floor2);
        const int myrot = in_smem ? jacobi_sweep_smem<T, NPL>(Z, p, n, 0, rt, f2, mycos)
                                  : jacobi_sweep_blocked<T, NPL>(Z, p, n, bs, slot, rt, f2, mycos);
        if (lane == 0 && myrot) atomicAdd(nrot_sh, myrot);
        {
            double mc = (double)mycos;
            for (int o = 16; o > 0; o >>= 1) mc = fmax(mc, __shfl_xor_sync(0xffffffffu, mc, o));
            if (lane == 0) atomicMax(maxcos_sh, (unsigned long long)__double_as_longlong(mc));
        }
        __syncthreads();
        const int total = *nrot_sh;
        const double mc = __longlong_as_double((long long)*maxcos_sh);
        __syncthreads();
        if (total == 0) return sweep + 1;
        if (sweep == max_sweeps - 1 && threadIdx.x == 0) {
            atomicOr(status, DEV_NONCONVERGED);
            if (dbg && atomicCAS(reinterpret_cast<unsigned long long*>(dbg), 0ull,
                                 (unsigned long long)__double_as_longlong((double)p)) == 0ull) {
                dbg[1] = n;
                dbg[2] = total;
                dbg[3] = mc;
            }
        }
    }
    return max_sweeps;
}

// One CTA per term.  Dynamic smem: Z (p*n*sizeof(T)) when it fits, plus
// p doubles (sigma^2) and p ints (order).
template <class T, int NPL>
__global__ void __launch_bounds__(256) k_jacobi_select(JacobiJob<T> job, int z_in_smem) {
    // z_in_smem: 1 = Z copied to shared memory; 0 = blocked ordering with Z in
    // global memory and a shared-memory slot of 2*job.blk rows
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int nrot_sh;
    __shared__ int kkeep_sh;
    __shared__ unsigned long long maxcos_sh;
    const int b = blockIdx.x;
    const int p = job.p, n = job.n, kout = job.kout;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    double* s2 = reinterpret_cast<double*>(smem_raw);
    int* order = reinterpret_cast<int*>(s2 + p);
    T* Zg = job.Z + (long)b * job.strideZ;
    T* Z = Zg;
    T* after = reinterpret_cast<T*>(smem_raw + ((p * (sizeof(double) + sizeof(int)) + 15) & ~15));
    if (z_in_smem) {
        Z = after;
        cta_copy(Z, Zg, (long)p * n);
        __syncthreads();
    }
    // Frobenius norm (invariant under the rotations) sets the rounding floor
    __shared__ double red[32];
    double part = 0.0;
    for (int i = tid; i < p * n; i += nt) {
        const double x = Z[i];
        part += x * x;
    }
    const double fro2 = block_sum(part, red);
    const double floor2 = Real<T>::eps * Real<T>::eps * fro2;
    const int sweeps = jacobi_rows<T, NPL>(Z, p, n, z_in_smem, job.blk, after, job.rot_tol, floor2,
                                           job.max_sweeps, &nrot_sh, &maxcos_sh, job.status, job.dbg);
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
    // squared row norms in float64
    for (int r = wid; r < p; r += nw) {
        double acc = 0.0;
        for (int c = lane; c < n; c += 32) {
            const double x = Z[(long)r * n + c];
            acc += x * x;
        }
        acc = warp_sum(acc);
        if (lane == 0) s2[r] = acc;
    }
    __syncthreads();
    // rank by descending sigma (ties by index): order[rank] = row
    for (int r = tid; r < p; r += nt) {
        const double v = s2[r];
        int rank = 0;
        for (int q = 0; q < p; ++q) {
            const double w = s2[q];
            rank += (w > v) || (w == v && q < r);
        }
        order[rank] = r;
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
    const double thresh = 2.0 * Real<T>::eps * sqrt(fro2);
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
        if (lane == 0) sv[j] = row >= 0 ? sig : 0.0;
        const double inv = row >= 0 ? 1.0 / sig : 0.0;
        const int* cm = job.colmap ? job.colmap + (long)b * n : nullptr;
        for (int c = lane; c < n; c += 32)
            V[(long)j * n + (cm ? cm[c] : c)] = row >= 0 ? T(Z[(long)row * n + c] * inv) : T(0);
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
    for (int r = 0; r < mU; ++r) {
        const double x = U[(long)r * kout + j];
        acc += x * x;
    }
    const double nrm = sqrt(acc);
    const T inv = nrm > 0.0 ? T(1.0 / nrm) : T(0);
    for (int r = 0; r < mU; ++r) U[(long)r * kout + j] *= inv;
    nu[(long)b * strideNu + j] = nrm > 0.0 ? T(nrm) : T(0);
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
        if (fii == T(0)) return T(0);  // dropped row: M row stays zero
        const T fp = (i == l) ? f - T(1) : f;
        return nu[(long)b * sNu + i] * ((i == l ? T(1) : T(0)) - fp);
    }
};

}  // namespace thc
