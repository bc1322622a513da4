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
    double* dbg;       // [4]: p, n, rotations and max cosine of the last sweep of the
                       // first matrix that did not converge (written once)
};

// player at tournament position `pos` in round r (position 0 fixed)
__device__ __forceinline__ int rr_player(int pos, int r, int P2) {
    return pos == 0 ? 0 : ((pos - 1 + r) % (P2 - 1)) + 1;
}

// Rows with ||z||^2 <= floor2 are numerically zero (below the rounding level of
// the matrix they came from): they are not rotated, and the selection drops them.
template <class T, int NPL>
__device__ void jacobi_rows(T* Z, int p, int n, double rot_tol, double floor2, int max_sweeps,
                            int* nrot_sh, unsigned long long* maxcos_sh, int* status, double* dbg) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int P2 = p + (p & 1);
    if (P2 < 2) return;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) {
            *nrot_sh = 0;
            *maxcos_sh = 0ull;
        }
        __syncthreads();
        int myrot = 0;
        double mycos = 0.0;
        for (int r = 0; r < P2 - 1; ++r) {
            for (int pi = wid; pi < P2 / 2; pi += nw) {
                int a = rr_player(pi, r, P2), bb = rr_player(P2 - 1 - pi, r, P2);
                if (a >= p || bb >= p) continue;
                T* za = Z + (long)a * n;
                T* zb = Z + (long)bb * n;
                T xa[NPL], xb[NPL];
                T al = 0, be = 0, ga = 0;
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int c = lane + 32 * i;
                    xa[i] = c < n ? za[c] : T(0);
                    xb[i] = c < n ? zb[c] : T(0);
                    al += xa[i] * xa[i];
                    be += xb[i] * xb[i];
                    ga += xa[i] * xb[i];
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                const double da = al, db = be, dg = ga;
                if (da <= floor2 || db <= floor2) continue;
                const double nab = sqrt(da) * sqrt(db);  // no underflow of da*db
                mycos = fmax(mycos, fabs(dg) / nab);
                if (fabs(dg) <= rot_tol * nab) continue;
                // rotation zeroing the (a,b) entry of the 2x2 Gram [[al, ga], [ga, be]]
                const double zeta = (db - da) / (2.0 * dg);
                const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + t * t);
                const T c = T(cs), s = T(cs * t);
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int col = lane + 32 * i;
                    if (col < n) {
                        const T na = c * xa[i] - s * xb[i];
                        const T nb = s * xa[i] + c * xb[i];
                        za[col] = na;
                        zb[col] = nb;
                    }
                }
                ++myrot;
            }
            __syncthreads();
        }
        if (lane == 0 && myrot) atomicAdd(nrot_sh, myrot);
        if (lane == 0) atomicMax(maxcos_sh, (unsigned long long)__double_as_longlong(mycos));
        __syncthreads();
        const int total = *nrot_sh;
        const double mc = __longlong_as_double((long long)*maxcos_sh);
        __syncthreads();
        if (total == 0) return;
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
}

// One CTA per term.  Dynamic smem: Z (p*n*sizeof(T)) when it fits, plus
// p doubles (sigma^2) and p ints (order).
template <class T, int NPL>
__global__ void __launch_bounds__(256) k_jacobi_select(JacobiJob<T> job, int z_in_smem) {
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
    if (z_in_smem) {
        Z = reinterpret_cast<T*>(smem_raw + ((p * (sizeof(double) + sizeof(int)) + 15) & ~15));
        for (int i = tid; i < p * n; i += nt) Z[i] = Zg[i];
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
    jacobi_rows<T, NPL>(Z, p, n, job.rot_tol, floor2, job.max_sweeps, &nrot_sh, &maxcos_sh, job.status,
                        job.dbg);
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
        for (int c = lane; c < n; c += 32)
            V[(long)j * n + c] = row >= 0 ? T(Z[(long)row * n + c] * inv) : T(0);
    }
}

// Finalisation per term: normalise the columns of U (mU x kout, row-major, in
// place) and write M = N (I - F) V (kout x n) with F = V V^T - I on the rows
// that are kept.  Dynamic smem: kout*kout T (F) + kout T (norms).
template <class T>
__global__ void __launch_bounds__(256)
k_svd_finalize(T* U, long strideU, int mU, const T* V, long strideV, int n, int kout,
               T* M, long strideM) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* F = reinterpret_cast<T*>(smem_raw);
    T* nu = F + (size_t)kout * kout;
    const int b = blockIdx.x;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    U += (long)b * strideU;
    V += (long)b * strideV;
    M += (long)b * strideM;
    for (int j = wid; j < kout; j += nw) {
        double acc = 0.0;
        for (int r = lane; r < mU; r += 32) {
            const double x = U[(long)r * kout + j];
            acc += x * x;
        }
        acc = warp_sum(acc);
        const double nrm = sqrt(acc);
        const T inv = nrm > 0.0 ? T(1.0 / nrm) : T(0);
        for (int r = lane; r < mU; r += 32) U[(long)r * kout + j] *= inv;
        if (lane == 0) nu[j] = nrm > 0.0 ? T(nrm) : T(0);
    }
    // F = V V^T - I (zero for rows that are zero)
    for (int o = tid; o < kout * kout; o += nt) {
        const int i = o / kout, j = o % kout;
        T s = 0;
        const T* vi = V + (long)i * n;
        const T* vj = V + (long)j * n;
        for (int c = 0; c < n; ++c) s += vi[c] * vj[c];
        F[o] = (i == j) ? (s != T(0) ? s - T(1) : T(0)) : s;
    }
    __syncthreads();
    for (int o = tid; o < kout * n; o += nt) {
        const int i = o / n, c = o % n;
        T s = V[(long)i * n + c];
        for (int l = 0; l < kout; ++l) s -= F[i * kout + l] * V[(long)l * n + c];
        M[o] = nu[i] * s;
    }
}

}  // namespace thc
