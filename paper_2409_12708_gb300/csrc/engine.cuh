// engine.cuh -- host orchestration of the THC-MPO hot path on one GPU.
//
// Data layout in HBM: a batch of B MPS with a common bond profile is one
// allocation, term-major: term b's site s starts at base + b*stride + off[s]
// and is [bond[s], 4, bond[s+1]] row-major.  All shapes are static (they follow
// from L, the input profile and D_max), so every launch of a sweep step covers
// the whole batch with one CTA (or one GEMM tile) per term.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <stdexcept>
#include <string>
#include <tuple>
#include <type_traits>
#include <typeinfo>
#include <vector>

#include "../../include/thc.h"
#include "common.cuh"
#include "gemm.cuh"
#include "scalar.cuh"
#include "jacobi.cuh"
#include "qr.cuh"
#include "qt_apply.cuh"
#include "small.cuh"
#include "terms.cuh"
#include "tc_gemm.cuh"

namespace thc {

// ----------------------------------------------------------------------------
// errors and memory
// ----------------------------------------------------------------------------
struct Error : std::runtime_error {
    thc_status st;
    Error(thc_status s, const std::string& m) : std::runtime_error(m), st(s) {}
};

#define THC_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            throw ::thc::Error(THC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct Alloc {
    const thc_allocator* a = nullptr;
    cudaStream_t st = nullptr;
    void* get(size_t bytes) const {
        if (bytes == 0) bytes = 16;
        void* p = nullptr;
        if (a && a->alloc) {
            p = a->alloc(bytes, (void*)st, a->ctx);
        } else if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (!p) throw Error(THC_ENOMEM, "allocation of " + std::to_string(bytes) + " bytes failed");
        return p;
    }
    void put(void* p) const {
        if (!p) return;
        if (a && a->free) a->free(p, (void*)st, a->ctx);
        else cudaFreeAsync(p, st);
    }
};

// Stream-ordered scratch released in reverse order when it goes out of scope.
struct Scratch {
    Alloc al;
    std::vector<void*> ptrs;
    explicit Scratch(const Alloc& a) : al(a) {}
    template <class X> X* get(size_t n) {
        void* p = al.get(n * sizeof(X));
        ptrs.push_back(p);
        return static_cast<X*>(p);
    }
    void release() {
        for (auto it = ptrs.rbegin(); it != ptrs.rend(); ++it) al.put(*it);
        ptrs.clear();
    }
    ~Scratch() { release(); }
};

// ----------------------------------------------------------------------------
// launch accounting: every kernel launch is counted; with profiling on, each
// launch is bracketed by CUDA events on its own stream and the durations are
// summed per kernel name when read.
// ----------------------------------------------------------------------------
struct Profiler {
    std::atomic<unsigned long long> launches{0};
    bool on = false;
    std::mutex mu;
    struct Rec {
        const char* name;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    std::map<std::string, std::pair<long, double>> acc;
    cudaEvent_t ev() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    void drain() {  // fold finished records into the per-name sums
        for (auto& r : recs) {
            cudaEventSynchronize(r.b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, r.a, r.b);
            auto& x = acc[r.name];
            x.first += 1;
            x.second += ms;
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
    }
};
inline Profiler& profiler() {
    static Profiler p;
    return p;
}

struct LaunchScope {
    Profiler::Rec rec{nullptr, nullptr, nullptr};
    cudaStream_t st;
    LaunchScope(const char* name, cudaStream_t s) : st(s) {
        Profiler& p = profiler();
        p.launches.fetch_add(1, std::memory_order_relaxed);
        if (p.on) {
            std::lock_guard<std::mutex> g(p.mu);
            rec.name = name;
            rec.a = p.ev();
            rec.b = p.ev();
            cudaEventRecord(rec.a, st);
        }
    }
    ~LaunchScope() {
        if (rec.name) {
            Profiler& p = profiler();
            std::lock_guard<std::mutex> g(p.mu);
            cudaEventRecord(rec.b, st);
            p.recs.push_back(rec);
            if (p.recs.size() > 4096) p.drain();
        }
    }
};
#define THC_CAT2(a, b) a##b
#define THC_CAT(a, b) THC_CAT2(a, b)
#define THC_LAUNCH(name, st) ::thc::LaunchScope THC_CAT(thc_launch_, __LINE__)(name, st)

// ----------------------------------------------------------------------------
// bond profiles
// ----------------------------------------------------------------------------
struct Profile {
    int L = 0;
    std::vector<int> bond;   // L+1
    std::vector<long> off;   // L site offsets (elements)
    long size = 0;
    Profile() = default;
    explicit Profile(const std::vector<int>& b) : L((int)b.size() - 1), bond(b), off(b.size() - 1) {
        size = 0;
        for (int s = 0; s < L; ++s) {
            off[s] = size;
            size += (long)bond[s] * 4 * bond[s + 1];
        }
    }
    long site_size(int s) const { return (long)bond[s] * 4 * bond[s + 1]; }
};

inline std::vector<int> full_profile(int L, int D) {
    std::vector<int> b(L + 1);
    for (int s = 0; s <= L; ++s) {
        long v = D;
        long l = 1, r = 1;
        for (int i = 0; i < s && l < D; ++i) l *= 4;
        for (int i = 0; i < L - s && r < D; ++i) r *= 4;
        v = std::min<long>(v, std::min(l, r));
        b[s] = (int)v;
    }
    return b;
}

// ----------------------------------------------------------------------------
// compression plan: the shape chain of one "expand + compress" (Fig. 3)
// ----------------------------------------------------------------------------
enum ExpandMode : int { MODE_LAYER = 0, MODE_DIRSUM = 1, MODE_PLAIN = 2 };

struct Plan {
    int L = 0, D = 0, mode = MODE_LAYER;
    std::vector<int> inA, inB;   // input bonds (B only for DIRSUM)
    std::vector<int> e;          // expanded bonds (MPO bond x MPS bond)
    std::vector<int> k;          // bonds after the QR sweep
    std::vector<int> out;        // bonds after the SVD sweep
    std::vector<long> woff;      // slot s: X_s [e[s] x 4 k[s+1]]
    long wsize = 0;
    long maxL = 0, maxC = 0, maxZ = 0, maxV = 0, maxTw = 0, maxKout = 0, maxQRm = 0;
    int maxP = 0, maxN = 0;
};

template <class T>
inline void qr_params(int m, int n, int& nb) {
    nb = sizeof(T) >= 8 ? 16 : 32;  // panel width (at most one warp of reflectors)
    const size_t budget = 220 * 1024;
    while (nb > 4 && qr_smem_bytes<T>(m, nb, n) > budget) nb /= 2;
    if (qr_smem_bytes<T>(m, nb, n) > budget)
        throw Error(THC_EUNSUPPORTED, "QR column length too large for shared memory");
}

template <class T>
inline Plan make_plan(int mode, const std::vector<int>& inA, const std::vector<int>& inB, int D) {
    Plan P;
    P.L = (int)inA.size() - 1;
    P.D = D;
    P.mode = mode;
    P.inA = inA;
    P.inB = inB;
    const int L = P.L;
    P.e.assign(L + 1, 1);
    for (int b = 1; b < L; ++b)
        P.e[b] = (mode == MODE_LAYER) ? 2 * inA[b] : (mode == MODE_DIRSUM ? inA[b] + inB[b] : inA[b]);
    P.k.assign(L + 1, 1);
    for (int s = L - 1; s >= 1; --s) P.k[s] = std::min(P.e[s], 4 * P.k[s + 1]);
    P.k[0] = 1;
    P.out.assign(L + 1, 1);
    for (int s = 0; s < L - 1; ++s) P.out[s + 1] = std::min(D, std::min(4 * P.out[s], P.k[s + 1]));
    P.woff.assign(L, 0);
    P.wsize = 0;
    for (int s = 0; s < L; ++s) {
        P.woff[s] = P.wsize;
        P.wsize += (long)P.e[s] * 4 * P.k[s + 1];
    }
    for (int s = 0; s < L; ++s) {
        P.maxL = std::max(P.maxL, (long)P.e[s] * P.k[s]);
        const int m = 4 * P.k[s + 1], n = P.e[s];
        if (s >= 1) {
            int nb;
            qr_params<T>(m, n, nb);
            P.maxTw = std::max(P.maxTw, (long)ceil_div(std::min(m, n), nb) * nb * nb);
            P.maxQRm = std::max<long>(P.maxQRm, m);
        }
    }
    for (int s = 0; s < L - 1; ++s) {
        const int m = 4 * P.out[s], n = P.k[s + 1];
        P.maxC = std::max(P.maxC, (long)m * n);
        const int p = std::min(m, n);
        P.maxZ = std::max(P.maxZ, (long)std::max(p, n) * n);
        P.maxV = std::max(P.maxV, (long)P.out[s + 1] * n);
        P.maxKout = std::max<long>(P.maxKout, P.out[s + 1]);
        P.maxP = std::max(P.maxP, p);
        P.maxN = std::max(P.maxN, n);
        if (m >= n) {
            int nb;
            qr_params<T>(m, n, nb);
            P.maxTw = std::max(P.maxTw, (long)ceil_div(n, nb) * nb * nb);
            P.maxQRm = std::max<long>(P.maxQRm, m);
        }
    }
    return P;
}

// ----------------------------------------------------------------------------
// device functors
// ----------------------------------------------------------------------------
// Local operators of App. C in the site basis n = 2 n_up + n_dn.  For each of
// the four ladder operators (o = sigma + 2*dagger) and output index n', the
// single input index n with a non-zero matrix element and its sign:
//   b_up = c (x) I2 : |up> -> |0>, |updn> -> |dn>
//   b_dn = Z (x) c  : |dn> -> |0>, |updn> -> -|up>
//   creation operators are the transposes.
static __constant__ signed char c_src[4][4] = {
    {2, 3, -1, -1},   // b_up   : n'=0 <- n=2, n'=1 <- n=3
    {1, -1, 3, -1},   // b_dn   : n'=0 <- n=1, n'=2 <- n=3
    {-1, -1, 0, 1},   // b_up^T : n'=2 <- n=0, n'=3 <- n=1
    {-1, 0, -1, 2},   // b_dn^T : n'=1 <- n=0, n'=3 <- n=2
};
static __constant__ signed char c_sgn[4][4] = {
    {1, 1, 0, 0},
    {1, 0, -1, 0},
    {0, 0, 1, 1},
    {0, 1, 0, -1},
};
// Jordan-Wigner string on one site, Z (x) Z = (-1)^(n_up + n_dn)
static __constant__ signed char c_par[4] = {1, -1, -1, 1};

// A-operand of the expand+absorb GEMM for site s: row m = (a_row, n'),
// column q = (b, beta) over the expanded right bond.
//   LAYER  (elementary MPO, Jordan-Wigner form of Sec. 3.1):
//     W[s] = [[Z(x)Z, coef_s b], [0, I4]]; site 1 keeps row a=0, site L column b=1.
//   DIRSUM (MPS addition): [A B] at site 1, diag(A, B) in the bulk, [A; B] at site L,
//     with the per-term coefficients on site 1.
//   PLAIN  (compression alone): the site itself.
template <class T>
struct ExpandA {
    int mode, s, L;
    const T* inA;
    long strideA;
    long offA;             // site offset in A's profile
    const int* srcA;       // per-term MPS index into inA (nullptr: term index)
    int lA, rA;            // A's bonds at site s
    const T* inB;
    long strideB;
    long offB;
    const int* srcB;
    int lB, rB;
    const T* coef;         // LAYER: coef[b*coef_ld + s]; DIRSUM: coefA[b], coefB[b] interleaved
    int coef_ld;
    const int* opsel;      // LAYER: per-term operator o = sigma + 2*dagger
    int rows0, cols0;      // size of the first row / column block

    __device__ __forceinline__ T operator()(int b, int m, int q) const {
        const int arow = m >> 2, np = m & 3;
        const int ai = arow < rows0 ? 0 : 1;
        const int alpha = arow - (ai ? rows0 : 0);
        const int bi = q < cols0 ? 0 : 1;
        const int beta = q - (bi ? cols0 : 0);
        if (mode == MODE_LAYER) {
            const int a = (s == 0) ? 0 : ai;
            const int bb = (s == L - 1) ? 1 : bi;
            const T* in = inA + (long)(srcA ? srcA[b] : b) * strideA + offA;
            if (a == 0 && bb == 0) return tscale(in[((long)alpha * 4 + np) * rA + beta], real_t<T>(c_par[np]));
            if (a == 1 && bb == 1) return in[((long)alpha * 4 + np) * rA + beta];
            if (a == 1 && bb == 0) return tzero<T>();
            const int o = opsel[b];
            const int n = c_src[o][np];
            if (n < 0) return tzero<T>();
            return coef[(long)b * coef_ld + s] *
                   tscale(in[((long)alpha * 4 + n) * rA + beta], real_t<T>(c_sgn[o][np]));
        }
        if (mode == MODE_PLAIN) {
            const T* in = inA + (long)(srcA ? srcA[b] : b) * strideA + offA;
            return in[((long)alpha * 4 + np) * rA + beta];
        }
        // DIRSUM
        int which;  // 0: A, 1: B, -1: zero
        if (s == 0) which = bi;
        else if (s == L - 1) which = ai;
        else which = (ai == bi) ? ai : -1;
        if (which < 0) return tzero<T>();
        if (which == 0) {
            const T* in = inA + (long)(srcA ? srcA[b] : b) * strideA + offA;
            const T v = in[((long)alpha * 4 + np) * rA + beta];
            return s == 0 ? coef[2 * b] * v : v;
        }
        const T* in = inB + (long)(srcB ? srcB[b] : b) * strideB + offB;
        const T v = in[((long)alpha * 4 + np) * rB + beta];
        return s == 0 ? coef[2 * b + 1] * v : v;
    }
};

template <class T>
struct RowMajorB {  // B(k, n) = base_b[k*ld + n]; identity 1x1 when base is null
    const T* base;
    long stride;
    int ld;
    __device__ __forceinline__ T operator()(int b, int k, int n) const {
        if (!base) return tone<T>();
        return base[(long)b * stride + (long)k * ld + n];
    }
};

template <class T>
struct RowMajorA {  // A(m, k) = base_b[m*ld + k]
    const T* base;
    long stride;
    int ld;
    __device__ __forceinline__ T operator()(int b, int m, int k) const {
        return base[(long)b * stride + (long)m * ld + k];
    }
};

template <class T>
struct TransB {  // B(k, n) = conj(base_b[n*ld + k]) (the conjugate transpose; real: transpose)
    const T* base;
    long stride;
    int ld;
    __device__ __forceinline__ T operator()(int b, int k, int n) const {
        return tconj(base[(long)b * stride + (long)n * ld + k]);
    }
};

template <class T>
struct StoreRM {  // C(m, n) -> base_b[m*ld + n]
    T* base;
    long stride;
    int ld;
    template <class A>
    __device__ __forceinline__ void operator()(int b, int m, int n, A v) const {
        base[(long)b * stride + (long)m * ld + n] = cvt<T>(v);
    }
};

template <class T>
struct StoreRMandCM {  // row-major C and a column-major copy (for the QR of C)
    T* rm;
    long srm;
    T* cm;
    long scm;
    int M, N;
    template <class A>
    __device__ __forceinline__ void operator()(int b, int m, int n, A v) const {
        rm[(long)b * srm + (long)m * N + n] = cvt<T>(v);
        if (cm) cm[(long)b * scm + (long)n * M + m] = cvt<T>(v);
    }
};

template <class T>
struct IdentA {  // the 1x1 identity (M_{-1} of the SVD sweep)
    __device__ __forceinline__ T operator()(int, int, int) const { return tone<T>(); }
};

// C of the SVD sweep, written row-major [(alpha, n') x j] and, when a QR of C
// follows, also column-major (GEMM row r = alpha, column col = (n', j)).
template <class T>
struct StoreC {
    T* rm;
    long srm;
    T* cm;
    long scm;
    int mC, nC, NG;
    template <class A>
    __device__ __forceinline__ void operator()(int b, int r, int col, A v) const {
        rm[(long)b * srm + (long)r * NG + col] = cvt<T>(v);
        if (cm) {
            const int row = r * 4 + col / nC, j = col % nC;
            cm[(long)b * scm + (long)j * mC + row] = cvt<T>(v);
        }
    }
};

// ----------------------------------------------------------------------------
// small kernels
// ----------------------------------------------------------------------------
template <class T, class S>
__global__ void k_copy_pad(T* dst, int dl, int dr, const S* src, int sl, int sr) {
    // dst [dl,4,dr] <- src [sl,4,sr] zero-padded (dl>=sl, dr>=sr), converted to T
    const long n = (long)dl * 4 * dr;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i % dr);
        const int np = (int)((i / dr) % 4);
        const int l = (int)(i / (4L * dr));
        dst[i] = (l < sl && r < sr) ? cvt<T>(src[((long)l * 4 + np) * sr + r]) : tzero<T>();
    }
}

template <class D, class S>
__global__ void k_convert(D* dst, const S* src, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = cvt<D>(src[i]);
}

template <class T>
__global__ void k_copy_batched(T* dst, long sdst, const T* src, long ssrc, long n) {
    const int b = blockIdx.y;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[(long)b * sdst + i] = src[(long)b * ssrc + i];
}

// Layer coefficients for a wave of terms (a1 of the hot path):
//  stage 0 (reuse, Alg. 1 lines for G_{nu s'}): term j = (nu, s'):
//      layer 1 = sum_s chi^nu_s a_{s s'}, layer 2 = sum_r chi^nu_r a+_{r s'}
//  stage 1 (per term t): Coulomb t -> (mu, s, nu, s'):
//      layer 1 = (zeta^{mu nu}/2) sum_q chi^mu_q a_{q s}, layer 2 = sum_p chi^mu_p a+_{p s},
//      source = reuse slot (s'*N + nu) - j_first;
//    kinetic t -> (i, s): layer 1 = lambda_i sum_q u_qi a_{q s}, layer 2 = sum_p u_pi a+_{p s},
//      source = 0 (psi itself).

template <class T>
__global__ void k_term_coefs(int stage, long t0, int B, int L, int N, int merge, const double* chi,
                             const double* zeta, const double* lam, const double* u,
                             long j_first, T* coef1, T* coef2, int* op1, int* op2, int* src) {
    const int b = blockIdx.x;
    if (b >= B) return;
    const long t = t0 + b;
    double scale = 1.0;
    int col = 0, sig = 0;
    bool kinetic = false;
    int source = 0;
    if (stage == 0) {
        const int nu = (int)(t % N), sp = (int)(t / N);  // reuse index j = s'*N + nu
        col = nu;
        sig = sp;
        source = 0;
    } else if (t < coulomb_terms(N, merge)) {
        const TermIdx d = decode_coulomb(t, N, merge);
        col = d.mu;
        sig = d.s;
        scale = d.factor * 0.5 * zeta[(long)d.mu * N + d.nu];
        source = (int)((long)d.sp * N + d.nu - j_first);
    } else {
        const long kk = t - coulomb_terms(N, merge);
        const int i = (int)(kk % L), s = (int)(kk / L);
        kinetic = true;
        col = i;
        sig = s;
        scale = lam[i];
        source = 0;
    }
    for (int s = threadIdx.x; s < L; s += blockDim.x) {
        const double c = kinetic ? u[(long)s * L + col] : chi[(long)s * N + col];
        coef1[(long)b * L + s] = cvt<T>(scale * c);
        coef2[(long)b * L + s] = cvt<T>(c);
    }
    if (threadIdx.x == 0) {
        op1[b] = sig;        // annihilation
        op2[b] = sig + 2;    // creation
        src[b] = source;
    }
}

template <class T>
__global__ void k_pair_coefs(T* coef, int B, const T* cA, const T* cB) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) {
        coef[2 * b] = cA ? cA[b] : tone<T>();
        coef[2 * b + 1] = cB ? cB[b] : tone<T>();
    }
}

}  // namespace thc
