// adjoint.cuh -- exact <phi|H|psi> and its derivatives with respect to t, chi,
// zeta and psi (the adjoint of the THC-MPO expectation value).
//
// Every term of H is a product of nl bond-2 ladder MPOs (Sec. 3.1): a Coulomb
// term G_{mu s, nu s'} = zeta^{mu nu} A+_{mu s} A_{mu s} A+_{nu s'} A_{nu s'}
// (Eq. G; four layers, A_{nu s'} applied first), a one-body term
// (sum_p t_pq a+_{p s}) a_{q s} (two layers, the first with coefficient e_q).
// A term's value <phi|W_{nl-1} ... W_0|psi> is contracted exactly (no
// compression) with environments over the composite MPO bond w in [0, 2^nl)
// (bit l = bond state of layer l):
//   left   E_{s+1}[a', w', b'] = sum phi_s[a, n', a'] M_s[w, w', n', n] E_s[a, w, b] psi_s[b, n, b']
//   right  R_s[a, w, b]       = sum phi_s[a, n', a'] M_s[w, w', n', n] R_{s+1}[a', w', b'] psi_s[b, n, b']
// with M_s the product of the layers' site-s tensors
// W = [[Z(x)Z, c_s b], [0, I4]] and boundary states w = 0 (left), w = all ones
// (right).  The derivatives follow from the two environments:
//   d value / d c^l_s = sum X_s[a, w, n, b'] (M'^l_s^T Q_s)[a, w, n, b'],
//       X_s = E_s psi_s, Q_s = phi_s R_{s+1}, M'^l_s = M_s with layer l's site-s
//       tensor replaced by dW/dc_s = [[0, b], [0, 0]];
//   d value / d psi_s = E_s^T (M_s^T Q_s).
// Each site is four batched GEMMs (the library's tiled GEMM) and two
// register-resident kernels that apply the layers (forward, or transposed
// with the coefficient gradients).  Real MPS only.
#pragma once

#include "common.cuh"
#include "scalar.cuh"

namespace thc {

// per-term layer data: nl layers, op[b*nl + l] = sigma + 2*dagger, coef[(b*nl + l)*L + s]
template <class T>
struct AdjTerms {
    const int* op;
    const T* coef;
    int nl, L;
};

// Layer l applied to the block Z[w][n] (2^NL x 4) at site s (input side bit l = a,
// output side bit l = b): Z'[b=0][n'] = par[n'] Z[a=0][n'],
// Z'[b=1][n'] = c sgn[n'] Z[a=0][src[n']] + Z[a=1][n'].
template <class T, int NL>
__device__ __forceinline__ void adj_layer_fwd(T (&Z)[1 << NL][4], int l, int o, T c) {
#pragma unroll
    for (int w = 0; w < (1 << NL); ++w) {
        if (w & (1 << l)) continue;
        const int w1 = w | (1 << l);
        T z0[4], z1[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            z0[n] = Z[w][n];
            z1[n] = Z[w1][n];
        }
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            Z[w][n] = T(c_par[n]) * z0[n];
            const int sidx = c_src[o][n];
            T v = z1[n];
            if (sidx >= 0) v += c * T(c_sgn[o][n]) * z0[sidx];
            Z[w1][n] = v;
        }
    }
}

// Transposed layer l on the output-side block Z[w'][n'] -> input side:
// Z'[a=0][n] = par[n] Z[b=0][n] + sum_{n': src[n'] = n} c sgn[n'] Z[b=1][n'],
// Z'[a=1][n] = Z[b=1][n].  deriv: the layer's derivative with respect to c
// (only the c b block, c = 1): Z'[a=0][n] = sum_{src[n'] = n} sgn[n'] Z[b=1][n'], Z'[a=1] = 0.
template <class T, int NL>
__device__ __forceinline__ void adj_layer_bwd(T (&Z)[1 << NL][4], int l, int o, T c, bool deriv) {
#pragma unroll
    for (int w = 0; w < (1 << NL); ++w) {
        if (w & (1 << l)) continue;
        const int w1 = w | (1 << l);
        T z0[4], z1[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            z0[n] = Z[w][n];
            z1[n] = Z[w1][n];
        }
        T a0[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) a0[n] = deriv ? T(0) : T(c_par[n]) * z0[n];
#pragma unroll
        for (int np = 0; np < 4; ++np) {
            const int sidx = c_src[o][np];
            if (sidx >= 0) a0[sidx] += (deriv ? T(1) : c) * T(c_sgn[o][np]) * z1[np];
        }
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            Z[w][n] = a0[n];
            Z[w1][n] = deriv ? T(0) : z1[n];
        }
    }
}

// Y[b][a][n'][w'][bp] = (M_s X)[...] for X[b][a][w][n][bp]; one thread per
// (a, bp), blockIdx.y = term b; sb = the buffers' stride between terms.
template <class T, int NL>
__global__ void k_adj_fwd(int Da, int Db, long sb, const T* X, T* Y, AdjTerms<T> tm, int s) {
    constexpr int NW = 1 << NL;
    const long per = (long)Da * Db;
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= per) return;
    const int b = blockIdx.y;
    const int a = (int)(idx / Db), bp = (int)(idx % Db);
    const T* x = X + (long)b * sb;
    T Z[NW][4];
#pragma unroll
    for (int w = 0; w < NW; ++w)
#pragma unroll
        for (int n = 0; n < 4; ++n) Z[w][n] = x[(((long)a * NW + w) * 4 + n) * Db + bp];
#pragma unroll
    for (int l = 0; l < NL; ++l) adj_layer_fwd<T, NL>(Z, l, tm.op[b * NL + l], tm.coef[((long)b * NL + l) * tm.L + s]);
    T* y = Y + (long)b * sb;
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int w = 0; w < NW; ++w) y[(((long)a * 4 + n) * NW + w) * Db + bp] = Z[w][n];
}

// P[b][a][w][n][bp] = (M_s^T Q)[...] for Q[b][a][n'][w'][bp]; with X given, also
// g[b][l][s] += sum X . (M'^l^T Q) (the coefficient gradients, reduced per block,
// one float64 atomic per block and layer).  One thread per (a, bp), blockIdx.y = b.
template <class T, int NL>
__global__ void __launch_bounds__(256) k_adj_bwd(int Da, int Db, long sb, const T* Q, T* P, const T* X, double* g,
                                                AdjTerms<T> tm, int s) {
    constexpr int NW = 1 << NL;
    __shared__ double red[NL][8];
    const long per = (long)Da * Db;
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const bool live = idx < per;
    const int b = blockIdx.y;
    const int a = live ? (int)(idx / Db) : 0, bp = live ? (int)(idx % Db) : 0;
    double part[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) part[l] = 0.0;
    if (live) {
        const T* q = Q + (long)b * sb;
        T Zq[NW][4];
#pragma unroll
        for (int n = 0; n < 4; ++n)
#pragma unroll
            for (int w = 0; w < NW; ++w) Zq[w][n] = q[(((long)a * 4 + n) * NW + w) * Db + bp];
        int ops[NL];
        T cs[NL];
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            ops[l] = tm.op[b * NL + l];
            cs[l] = tm.coef[((long)b * NL + l) * tm.L + s];
        }
        {
            T Z[NW][4];
#pragma unroll
            for (int w = 0; w < NW; ++w)
#pragma unroll
                for (int n = 0; n < 4; ++n) Z[w][n] = Zq[w][n];
#pragma unroll
            for (int l = NL - 1; l >= 0; --l) adj_layer_bwd<T, NL>(Z, l, ops[l], cs[l], false);
            T* p = P + (long)b * sb;
#pragma unroll
            for (int w = 0; w < NW; ++w)
#pragma unroll
                for (int n = 0; n < 4; ++n) p[(((long)a * NW + w) * 4 + n) * Db + bp] = Z[w][n];
        }
        if (X) {
            const T* x = X + (long)b * sb;
            T Zx[NW][4];
#pragma unroll
            for (int w = 0; w < NW; ++w)
#pragma unroll
                for (int n = 0; n < 4; ++n) Zx[w][n] = x[(((long)a * NW + w) * 4 + n) * Db + bp];
#pragma unroll
            for (int dl = 0; dl < NL; ++dl) {
                T Z[NW][4];
#pragma unroll
                for (int w = 0; w < NW; ++w)
#pragma unroll
                    for (int n = 0; n < 4; ++n) Z[w][n] = Zq[w][n];
#pragma unroll
                for (int l = NL - 1; l >= 0; --l) adj_layer_bwd<T, NL>(Z, l, ops[l], cs[l], l == dl);
                double d = 0.0;
#pragma unroll
                for (int w = 0; w < NW; ++w)
#pragma unroll
                    for (int n = 0; n < 4; ++n) d += (double)Zx[w][n] * (double)Z[w][n];
                part[dl] = d;
            }
        }
    }
    if (X) {  // block-uniform branch
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const double v = warp_sum(part[l]);
            if (lane == 0) red[l][wid] = v;
        }
        __syncthreads();
        if (threadIdx.x < NL) {
            double v = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
            atomicAdd(&g[((long)b * NL + threadIdx.x) * tm.L + s], v);
        }
    }
}

// The value of every term: E_L[b][0][NW-1][0].
template <class T>
__global__ void k_adj_values(int B, const T* EL, long strideE, int NW, double* val) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) val[b] = (double)EL[(long)b * strideE + (NW - 1)];
}

// boundary environments: E_0[b][0][0][0] = 1 (w = 0); R_L[b][0][NW-1][0] = 1
template <class T>
__global__ void k_adj_boundary(int B, T* E0, long sE, T* RL, long sR, int NW) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    for (int w = 0; w < NW; ++w) {
        E0[(long)b * sE + w] = T(w == 0 ? 1 : 0);
        RL[(long)b * sR + w] = T(w == NW - 1 ? 1 : 0);
    }
}

// dpsi_s += sum_b weight_b G[b] (one site, n elements per term, terms sg apart)
template <class T>
__global__ void k_adj_accum_site(int B, const T* G, long sg, long n, const double* weight, T* out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < B; ++b) acc += weight[b] * (double)G[(long)b * sg + i];
        out[i] = T((double)out[i] + acc);
    }
}

// The terms of H as layers.  kind 0 (one-body, 2L terms): j -> (q = j % L,
// s = j / L): layer 0 = a_{q s} (coefficient e_q), layer 1 = sum_p t_pq a+_{p s};
// weight 1.  kind 1 (Coulomb, 4N^2 terms, index ((s'N + nu)2 + s)N + mu):
// layers A_{nu s'}, A+_{nu s'}, A_{mu s}, A+_{mu s} (coefficients chi^nu, chi^nu,
// chi^mu, chi^mu); weight zeta^{mu nu} / 2.
template <class T>
__global__ void k_adj_terms(int kind, long t0, int B, int L, int N, const double* t, const double* chi,
                            const double* zeta, int* op, T* coef, double* weight) {
    const int b = blockIdx.x;
    if (b >= B) return;
    const long tt = t0 + b;
    if (kind == 0) {
        const int q = (int)(tt % L), sg = (int)(tt / L);
        for (int s = threadIdx.x; s < L; s += blockDim.x) {
            coef[((long)b * 2 + 0) * L + s] = T(s == q ? 1.0 : 0.0);
            coef[((long)b * 2 + 1) * L + s] = T(t[(long)s * L + q]);
        }
        if (threadIdx.x == 0) {
            op[b * 2 + 0] = sg;
            op[b * 2 + 1] = sg + 2;
            weight[b] = 1.0;
        }
    } else {
        const int mu = (int)(tt % N);
        long rest = tt / N;
        const int sg = (int)(rest % 2);
        rest /= 2;
        const int nu = (int)(rest % N), sp = (int)(rest / N);
        for (int s = threadIdx.x; s < L; s += blockDim.x) {
            const double cn = chi[(long)s * N + nu], cm = chi[(long)s * N + mu];
            coef[((long)b * 4 + 0) * L + s] = T(cn);
            coef[((long)b * 4 + 1) * L + s] = T(cn);
            coef[((long)b * 4 + 2) * L + s] = T(cm);
            coef[((long)b * 4 + 3) * L + s] = T(cm);
        }
        if (threadIdx.x == 0) {
            op[b * 4 + 0] = sp;
            op[b * 4 + 1] = sp + 2;
            op[b * 4 + 2] = sg;
            op[b * 4 + 3] = sg + 2;
            weight[b] = 0.5 * zeta[(long)mu * N + nu];
        }
    }
}

// Fold a batch of terms into the value and the parameter gradients (float64
// atomics): value += w_b v_b; kind 0: dt[p][q] += g[b][1][p]; kind 1:
// dzeta[mu][nu] += v_b / 2, dchi[s][nu] += w_b (g0 + g1)[s], dchi[s][mu] += w_b (g2 + g3)[s].
static __global__ void k_adj_params(int kind, long t0, int B, int L, int N, const double* val, const double* g,
                             const double* weight, double* value, double* dt, double* dchi, double* dzeta) {
    const int b = blockIdx.x;
    if (b >= B) return;
    const long tt = t0 + b;
    const double w = weight[b], v = val[b];
    if (threadIdx.x == 0) atomicAdd(value, w * v);
    if (kind == 0) {
        const int q = (int)(tt % L);
        if (dt)
            for (int p = threadIdx.x; p < L; p += blockDim.x) atomicAdd(&dt[(long)p * L + q], g[((long)b * 2 + 1) * L + p]);
    } else {
        const int mu = (int)(tt % N);
        const int nu = (int)((tt / (2L * N)) % N);
        if (dzeta && threadIdx.x == 0) atomicAdd(&dzeta[(long)mu * N + nu], 0.5 * v);
        if (dchi)
            for (int s = threadIdx.x; s < L; s += blockDim.x) {
                const double* gb = g + (long)b * 4 * L;
                atomicAdd(&dchi[(long)s * N + nu], w * (gb[0 * L + s] + gb[1 * L + s]));
                atomicAdd(&dchi[(long)s * N + mu], w * (gb[2 * L + s] + gb[3 * L + s]));
            }
    }
}

}  // namespace thc
