// engine_ops.cuh -- the library's operations built on Engine<T>.
#pragma once

#include <cmath>

#include "engine_impl.cuh"
#include "adjoint.cuh"

namespace thc {

// ---------------------------------------------------------------- inner product functors
// Transfer matrices are accumulated in Acc = Wide<T>: float64, or complex
// float64 for complex MPS.
template <class Acc>
struct EA {  // E(m, k), row-major
    const Acc* E;
    long sE;
    int ld;
    __device__ __forceinline__ Acc operator()(int b, int m, int k) const {
        return E[(long)b * sE + (long)m * ld + k];
    }
};
template <class T>
struct SiteB {  // B(k, n) = site[k*ld + n] of term b
    const T* base;
    long stride;
    int ld;
    __device__ __forceinline__ typename Wide<T>::type operator()(int b, int k, int n) const {
        return cvt<typename Wide<T>::type>(base[(long)b * stride + (long)k * ld + n]);
    }
};
template <class T>
struct SiteAT {  // A(m, k) = conj(site[k*ld + m]) (transposed access, conjugated: <phi| side)
    const T* base;
    long stride;
    int ld;
    __device__ __forceinline__ typename Wide<T>::type operator()(int b, int m, int k) const {
        return cvt<typename Wide<T>::type>(tconj(base[(long)b * stride + (long)k * ld + m]));
    }
};
template <class Acc>
struct StoreD {
    Acc* base;
    long stride;
    int ld;
    __device__ __forceinline__ void operator()(int b, int m, int n, Acc v) const {
        base[(long)b * stride + (long)m * ld + n] = v;
    }
};

template <class Acc>
__global__ void k_set_one(Acc* E, long stride, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) E[(long)b * stride] = tone<Acc>();
}
template <class Acc>
__global__ void k_gather_scalar(const Acc* E, long stride, int B, Acc* out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) out[b] = E[(long)b * stride];
}
// x <- c x with a float64 (complex float64) coefficient
template <class T>
__global__ void k_scale(T* x, long n, typename Wide<T>::type c) {
    using Acc = typename Wide<T>::type;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        x[i] = cvt<T>(cvt<Acc>(x[i]) * c);
}

static __global__ void k_set_int(int* p, int v) { *p = v; }

template <class T>
struct AdjTransA {  // A(m, k) = base_b[k*ld + m] (transposed access, real)
    const T* base;
    long stride;
    int ld;
    __device__ __forceinline__ T operator()(int b, int m, int k) const {
        return base[(long)b * stride + (long)k * ld + m];
    }
};

static __global__ void k_pack_complex(c64* out, const double* re, const double* im, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = c64{re[i], im[i]};
}

// A device MPS in the engine's contiguous layout (one term).
template <class T>
struct DevMps {
    T* base = nullptr;
    std::vector<int> bond;
};

template <class T>
struct Ops {
    using Acc = typename Wide<T>::type;  // float64 accumulator (complex for complex T)
    Engine<T>& E;
    explicit Ops(Engine<T>& e) : E(e) {}
    cudaStream_t st() const { return E.st; }

    // ------------------------------------------------------------- transfers
    // copy (zero-padded to prof) a caller's MPS; a real MPS given to a complex
    // engine is converted on the way
    void upload(const thc_mps* m, const std::vector<int>& prof, T* dst) {
        Profile p(prof);
        const bool widen = is_complex_v<T> && (m->dtype == THC_F64 || m->dtype == THC_F32);
        for (int s = 0; s < m->L; ++s) {
            const long n = p.site_size(s);
            const int blocks = std::max(1, (int)std::min<long>(ceil_div((int)std::min<long>(n, 1L << 30), 256), 4096));
            THC_LAUNCH("copy", st());
            if constexpr (is_complex_v<T>) {
                if (widen) {
                    k_copy_pad<T, real_t<T>><<<blocks, 256, 0, st()>>>(dst + p.off[s], prof[s], prof[s + 1],
                                                                         (const real_t<T>*)m->site[s], m->bond[s],
                                                                         m->bond[s + 1]);
                    E.check();
                    continue;
                }
            }
            k_copy_pad<T, T><<<blocks, 256, 0, st()>>>(dst + p.off[s], prof[s], prof[s + 1], (const T*)m->site[s],
                                                       m->bond[s], m->bond[s + 1]);
            E.check();
        }
    }

    void download(const T* src, const std::vector<int>& prof, thc_mps* out, thc_dtype dt) {
        Profile p(prof);
        void* blk = E.al.get((size_t)p.size * sizeof(T));
        THC_CUDA(cudaMemcpyAsync(blk, src, p.size * sizeof(T), cudaMemcpyDeviceToDevice, st()));
        std::memset(out, 0, sizeof(*out));
        out->L = p.L;
        out->d = 4;
        out->dtype = dt;
        for (int b = 0; b <= p.L; ++b) out->bond[b] = prof[b];
        for (int s = 0; s < p.L; ++s) out->site[s] = (void*)((T*)blk + p.off[s]);
        out->owner = blk;
    }

    // --------------------------------------------------------- inner products
    // <phi_b|psi_b> for B pairs stored strided (phi: base + b*sphi, psi: base + b*spsi).
    void inner_batched(int B, const T* phi, long sphi, const std::vector<int>& pp, const T* psi,
                       long spsi, const std::vector<int>& pq, Acc* out_dev) {
        Profile a(pp), c(pq);
        const int L = a.L;
        int ma = 1, mb = 1;
        for (int x : pp) ma = std::max(ma, x);
        for (int x : pq) mb = std::max(mb, x);
        Scratch sc(E.al);
        const long sE = (long)ma * mb, sF = (long)ma * 4 * mb;
        Acc* Eb = sc.get<Acc>((size_t)B * sE);
        Acc* Fb = sc.get<Acc>((size_t)B * sF);
        {
            THC_LAUNCH("setup", st());
            k_set_one<Acc><<<ceil_div(B, 128), 128, 0, st()>>>(Eb, sE, B);
        }
        E.check();
        for (int s = 0; s < L; ++s) {
            const int al = pp[s], ar = pp[s + 1], bl = pq[s], br = pq[s + 1];
            // F = E B_s  : [al x bl] x [bl x 4 br]
            {
            THC_LAUNCH("gemm_inner", st());
            THC_CUDA(launch_gemm<Acc>(B, al, 4 * br, bl, EA<Acc>{Eb, sE, bl},
                                      SiteB<T>{psi + c.off[s], spsi, 4 * br}, StoreD<Acc>{Fb, sF, 4 * br}, st()));
            }
            // E' = A_s^T F : [(al,4) x ar]^T x [(al,4) x br]
            {
            THC_LAUNCH("gemm_inner", st());
            THC_CUDA(launch_gemm<Acc>(B, ar, br, 4 * al, SiteAT<T>{phi + a.off[s], sphi, ar},
                                      EA<Acc>{Fb, sF, br}, StoreD<Acc>{Eb, sE, br}, st()));
            }
        }
        {
            THC_LAUNCH("setup", st());
            k_gather_scalar<Acc><<<ceil_div(B, 128), 128, 0, st()>>>(Eb, sE, B, out_dev);
        }
        E.check();
    }

    Acc inner1(const T* phi, const std::vector<int>& pp, const T* psi, const std::vector<int>& pq) {
        Scratch sc(E.al);
        Acc* d = sc.get<Acc>(1);
        inner_batched(1, phi, 0, pp, psi, 0, pq, d);
        Acc h = tzero<Acc>();
        THC_CUDA(cudaMemcpyAsync(&h, d, sizeof(Acc), cudaMemcpyDeviceToHost, st()));
        THC_CUDA(cudaStreamSynchronize(st()));
        return h;
    }

    // ------------------------------------------------------------ layer apply
    void layer_apply(const T* psi, const std::vector<int>& pin, const double* coef_dev, int sigma,
                     int dagger, int D, T* out, std::vector<int>& pout, int Bw) {
        Plan P = make_plan<T>(MODE_LAYER, pin, {}, D);
        Scratch sc(E.al);
        Work<T> w;
        E.alloc_work(sc, w, 1, {&P});
        const int L = P.L;
        {
            THC_LAUNCH("setup", st());
            k_convert<T, double><<<1, 64, 0, st()>>>(w.coef1, coef_dev, L);
        }
        const int op = sigma + 2 * (dagger ? 1 : 0);
        {
            THC_LAUNCH("setup", st());
            k_set_int<<<1, 1, 0, st()>>>(w.op1, op);
        }
        E.check();
        ExpandA<T> ex{};
        ex.mode = MODE_LAYER;
        ex.inA = psi;
        ex.strideA = 0;
        ex.coef = w.coef1;
        ex.coef_ld = L;
        ex.opsel = w.op1;
        E.compress(P, 1, ex, out, 0, w);
        pout = P.out;
    }

    void plain_compress(const T* psi, const std::vector<int>& pin, int D, T* out, std::vector<int>& pout) {
        Plan P = make_plan<T>(MODE_PLAIN, pin, {}, D);
        Scratch sc(E.al);
        Work<T> w;
        E.alloc_work(sc, w, 1, {&P});
        ExpandA<T> ex{};
        ex.mode = MODE_PLAIN;
        ex.inA = psi;
        E.compress(P, 1, ex, out, 0, w);
        pout = P.out;
    }

    // --------------------------------------------------------------- H|psi>
    // psi: device MPS with profile pin (every bond >= the full profile of D).
    // Output written to out (profile full_profile(L, D)).
    void apply_H(const thc_hamiltonian* H, const T* psi, const std::vector<int>& pin, const thc_opts* o,
                 T* out) {
        const int L = H->L, N = H->N, D = o->D_max;
        const std::vector<int> pf = full_profile(L, D);
        Profile Pf(pf);
        Scratch sc(E.al);
        E.tol_ = o->tol;
        double* lam = sc.get<double>(L);
        double* u = sc.get<double>((size_t)L * L);
        {
            THC_LAUNCH("kinetic_eigh", st());
            k_kinetic_factors<<<1, 256, KINETIC_SMEM, st()>>>(L, H->t, lam, u, E.dflag);
        }
        E.check();
        const int merge = o->merge_spin ? 1 : 0;
        const long VV = coulomb_terms(N, merge);
        const long TT = VV + 2L * L;
        const long t0 = std::max(0L, o->term_begin < 0 ? 0L : o->term_begin);
        const long t1 = (o->term_end < 0) ? TT : std::min(TT, o->term_end);
        const long nT = t1 - t0;
        if (nT <= 0) throw Error(THC_EINVAL, "empty term range");
        Plan PA1 = make_plan<T>(MODE_LAYER, pin, {}, D);
        Plan PA2 = make_plan<T>(MODE_LAYER, PA1.out, {}, D);
        Plan PB1 = make_plan<T>(MODE_LAYER, pf, {}, D);
        Plan PB2 = make_plan<T>(MODE_LAYER, PB1.out, {}, D);
        Plan PD = make_plan<T>(MODE_DIRSUM, pf, pf, D);
        if (PA2.out != pf || PB2.out != pf || PD.out != pf)
            throw Error(THC_EINVAL, "input bonds below the full profile of D_max");
        const long cEnd = std::min(t1, VV);
        const bool hasV = t0 < cEnd;
        // the reused states psi_{nu s'} the range needs: blocks are contiguous in
        // the term order (both lists), so they are the slots j_first .. j_last
        const long j_first = hasV ? coulomb_block(t0, N, merge) : 0;
        const long nslots = hasV ? coulomb_block(cEnd - 1, N, merge) - j_first + 1 : 0;
        // batch (terms in flight)
        const std::vector<const Plan*> plans{&PA1, &PA2, &PB1, &PB2, &PD};
        const size_t per_term = Engine<T>::work_bytes_per_term(plans) +
                                sizeof(T) * (size_t)std::max(Profile(PA1.out).size, Profile(PB1.out).size);
        size_t freeb = 0, totalb = 0;
        THC_CUDA(cudaMemGetInfo(&freeb, &totalb));
        long Bw = o->batch > 0 ? o->batch : 4L * E.sms;
        Bw = std::max(1L, std::min<long>(Bw, (long)(0.3 * freeb / std::max<size_t>(per_term, 1))));
        Bw = std::min<long>(Bw, std::max(nT, nslots));
        Scratch sw(E.al);
        Work<T> w;
        E.alloc_work(sw, w, (int)Bw, plans);
        T* tmp = sw.get<T>((size_t)Bw * std::max(Profile(PA1.out).size, Profile(PB1.out).size));
        T* reuse = hasV ? sc.get<T>((size_t)nslots * Pf.size) : nullptr;
        // ---- reuse stage (Alg. 1): psi_{nu s'} = compress(A+ compress(A psi))
        for (long j0 = 0; j0 < nslots; j0 += Bw) {
            const int Bc = (int)std::min<long>(Bw, nslots - j0);
            {
                THC_LAUNCH("term_coefs", st());
                k_term_coefs<T><<<Bc, 64, 0, st()>>>(0, j_first + j0, Bc, L, N, merge, H->chi, H->zeta, lam, u,
                                                      j_first, w.coef1, w.coef2, w.op1, w.op2, w.src);
            }
            E.check();
            ExpandA<T> e1{};
            e1.mode = MODE_LAYER;
            e1.inA = psi;
            e1.strideA = 0;
            e1.srcA = w.src;
            e1.coef = w.coef1;
            e1.coef_ld = L;
            e1.opsel = w.op1;
            E.compress(PA1, Bc, e1, tmp, Profile(PA1.out).size, w);
            ExpandA<T> e2 = e1;
            e2.inA = tmp;
            e2.strideA = Profile(PA1.out).size;
            e2.srcA = nullptr;
            e2.coef = w.coef2;
            e2.opsel = w.op2;
            E.compress(PA2, Bc, e2, reuse + j0 * Pf.size, Pf.size, w);
        }
        // ---- terms, in power-of-two chunks that are exact subtrees of the pairwise reduction
        THC_CUDA(cudaMemGetInfo(&freeb, &totalb));
        long chunk = 1;
        while (chunk < nT && (double)(2 * chunk) * 1.8 * Pf.size * sizeof(T) < 0.5 * freeb &&
               (o->chunk <= 0 || 2 * chunk <= o->chunk))
            chunk *= 2;
        const long nchunks = (nT + chunk - 1) / chunk;
        T* chunkres = sc.get<T>((size_t)nchunks * Pf.size);
        for (long ci = 0; ci < nchunks; ++ci) {
            const long c0 = ci * chunk, c1 = std::min(nT, c0 + chunk), n = c1 - c0;
            Scratch scc(E.al);
            T* res = scc.get<T>((size_t)n * Pf.size);
            long w0 = c0;
            while (w0 < c1) {
                const long t = t0 + w0;
                const bool isV = t < VV;
                long w1 = std::min(c1, w0 + Bw);
                if (isV) w1 = std::min(w1, VV - t0);
                const int Bc = (int)(w1 - w0);
                {
                    THC_LAUNCH("term_coefs", st());
                    k_term_coefs<T><<<Bc, 64, 0, st()>>>(1, t, Bc, L, N, merge, H->chi, H->zeta, lam, u, j_first,
                                                          w.coef1, w.coef2, w.op1, w.op2, w.src);
                }
                E.check();
                const Plan& P1 = isV ? PB1 : PA1;
                const Plan& P2 = isV ? PB2 : PA2;
                ExpandA<T> e1{};
                e1.mode = MODE_LAYER;
                e1.inA = isV ? reuse : psi;
                e1.strideA = isV ? Pf.size : 0;
                e1.srcA = w.src;
                e1.coef = w.coef1;
                e1.coef_ld = L;
                e1.opsel = w.op1;
                const long s1 = Profile(P1.out).size;
                E.compress(P1, Bc, e1, tmp, s1, w);
                ExpandA<T> e2 = e1;
                e2.inA = tmp;
                e2.strideA = s1;
                e2.srcA = nullptr;
                e2.coef = w.coef2;
                e2.opsel = w.op2;
                E.compress(P2, Bc, e2, res + (w0 - c0) * Pf.size, Pf.size, w);
                w0 = w1;
            }
            T* r = E.reduce(scc, res, n, pf, D, (int)Bw);
            THC_CUDA(cudaMemcpyAsync(chunkres + ci * Pf.size, r, Pf.size * sizeof(T),
                                     cudaMemcpyDeviceToDevice, st()));
        }
        T* fin = E.reduce(sc, chunkres, nchunks, pf, D, (int)Bw);
        THC_CUDA(cudaMemcpyAsync(out, fin, Pf.size * sizeof(T), cudaMemcpyDeviceToDevice, st()));
    }

    // ------------------------------------------------------ add and compress
    // sum_i c_i x_i (all with profile pf, the full profile of D) by the pairwise reduction.
    void add_compress(int n, const Acc* c, const T* const* xs, const std::vector<int>& pf, int D,
                      T* out) {
        Profile P(pf);
        Scratch sc(E.al);
        T* buf = sc.get<T>((size_t)n * P.size);
        for (int i = 0; i < n; ++i) {
            THC_CUDA(cudaMemcpyAsync(buf + (long)i * P.size, xs[i], P.size * sizeof(T),
                                     cudaMemcpyDeviceToDevice, st()));
            const long s = P.L - 1;
            {
                THC_LAUNCH("scale", st());
                k_scale<T><<<64, 256, 0, st()>>>(buf + (long)i * P.size + P.off[s], P.site_size(s), c[i]);
            }
            E.check();
        }
        T* r = E.reduce(sc, buf, n, pf, D, std::max(1, std::min(n / 2, 4 * E.sms)));
        THC_CUDA(cudaMemcpyAsync(out, r, P.size * sizeof(T), cudaMemcpyDeviceToDevice, st()));
    }

    // ------------------------------------------------------------- Lanczos
    // Returns the number of Krylov vectors; Ht, S (n x n host, row-major).
    // lower: optional orthonormal states (profile pf) the start vector and
    // every Krylov vector are orthogonalised against, in the same Gram-Schmidt
    // sum (excited states).
    int krylov_basis(const thc_hamiltonian* H, const T* psi0, const std::vector<int>& pf, int K,
                     const thc_opts* o, T* vbuf, T* wbuf, std::vector<Acc>& Ht,
                     std::vector<Acc>& S, const std::vector<const T*>& lower = {}) {
        Profile P(pf);
        const long sz = P.size;
        const int nl = (int)lower.size();
        if (nl > 0) {
            // v_0 = psi0 - sum_m <phi_m|psi0> phi_m
            std::vector<const T*> xs{psi0};
            std::vector<Acc> cs{tone<Acc>()};
            for (int m = 0; m < nl; ++m) {
                xs.push_back(lower[m]);
                cs.push_back(tzero<Acc>() - inner1(lower[m], pf, psi0, pf));
            }
            add_compress((int)xs.size(), cs.data(), xs.data(), pf, o->D_max, vbuf);
        } else {
            THC_CUDA(cudaMemcpyAsync(vbuf, psi0, sz * sizeof(T), cudaMemcpyDeviceToDevice, st()));
        }
        const double n0 = std::sqrt(std::fabs(treal_part(inner1(vbuf, pf, vbuf, pf))));
        if (!(n0 > 0.0)) throw Error(THC_EBREAKDOWN, "zero initial vector");
        {
            THC_LAUNCH("scale", st());
            k_scale<T><<<64, 256, 0, st()>>>(vbuf + P.off[P.L - 1], P.site_size(P.L - 1), cvt<Acc>(1.0 / n0));
        }
        E.check();
        int nv = 1;
        Scratch sc(E.al);
        Acc* hd = sc.get<Acc>((size_t)K + 1);
        for (int k = 0; k < K; ++k) {
            apply_H(H, vbuf + k * sz, pf, o, wbuf + k * sz);
            if (k == K - 1) break;
            inner_batched(k + 1, vbuf, sz, pf, wbuf + k * sz, 0, pf, hd);
            std::vector<Acc> h(k + 1);
            THC_CUDA(cudaMemcpyAsync(h.data(), hd, (k + 1) * sizeof(Acc), cudaMemcpyDeviceToHost, st()));
            THC_CUDA(cudaStreamSynchronize(st()));
            std::vector<const T*> xs;
            std::vector<Acc> cs;
            xs.push_back(wbuf + k * sz);
            cs.push_back(tone<Acc>());
            for (int j = 0; j <= k; ++j) {
                xs.push_back(vbuf + j * sz);
                cs.push_back(tzero<Acc>() - h[j]);
            }
            for (int m = 0; m < nl; ++m) {
                xs.push_back(lower[m]);
                cs.push_back(tzero<Acc>() - inner1(lower[m], pf, wbuf + k * sz, pf));
            }
            T* r = vbuf + (k + 1) * sz;
            add_compress((int)xs.size(), cs.data(), xs.data(), pf, o->D_max, r);
            const double nr = std::sqrt(std::fabs(treal_part(inner1(r, pf, r, pf))));
            const double nw = std::sqrt(std::fabs(treal_part(inner1(wbuf + k * sz, pf, wbuf + k * sz, pf))));
            if (!(nr >= 1e-8 * nw)) break;
            {
                THC_LAUNCH("scale", st());
                k_scale<T><<<64, 256, 0, st()>>>(r + P.off[P.L - 1], P.site_size(P.L - 1), cvt<Acc>(1.0 / nr));
            }
            E.check();
            nv = k + 2;
        }
        Ht.assign((size_t)nv * nv, tzero<Acc>());
        S.assign((size_t)nv * nv, tzero<Acc>());
        // columns k of Htil and S land in one device array (column-major), read back once
        Acc* cols = sc.get<Acc>((size_t)2 * nv * nv);
        for (int k = 0; k < nv; ++k) {
            inner_batched(nv, vbuf, sz, pf, wbuf + k * sz, 0, pf, cols + (size_t)k * nv);
            inner_batched(nv, vbuf, sz, pf, vbuf + k * sz, 0, pf, cols + (size_t)(nv + k) * nv);
        }
        std::vector<Acc> tmp((size_t)2 * nv * nv);
        THC_CUDA(cudaMemcpyAsync(tmp.data(), cols, tmp.size() * sizeof(Acc), cudaMemcpyDeviceToHost, st()));
        THC_CUDA(cudaStreamSynchronize(st()));
        for (int k = 0; k < nv; ++k)
            for (int j = 0; j < nv; ++j) {
                Ht[(size_t)j * nv + k] = tmp[(size_t)k * nv + j];
                S[(size_t)j * nv + k] = tmp[(size_t)(nv + k) * nv + j];
            }
        return nv;
    }

    // ------------------------------------------------------------- adjoint
    // value = <phi|H|psi> (exact, no compression) and, where the pointers are
    // given, dE/dt [L*L], dE/dchi [L*N], dE/dzeta [N*N] (device float64, added
    // to) and dE/dpsi (device, psi's profile, added to).  phi, psi: device MPS
    // in the contiguous layout with profiles pa, pb.  Real T only.
    void expect_grad(const thc_hamiltonian* H, const T* phi, const std::vector<int>& pa, const T* psi,
                     const std::vector<int>& pb, int batch, long term_begin, long term_end, double* value_dev,
                     double* dt, double* dchi, double* dzeta, T* dpsi) {
        static_assert(!is_complex_v<T>, "the adjoint is built for real MPS");
        const int L = H->L, N = H->N;
        Profile A(pa), Bp(pb);
        // the term range in thc_apply_H's indexing: Coulomb [0, 4N^2), one-body after
        const long VV = 4L * N * N, TT = VV + 2L * L;
        const long r0 = term_begin < 0 ? 0 : term_begin, r1 = term_end < 0 ? TT : std::min(TT, term_end);
        if (r1 <= r0) throw Error(THC_EINVAL, "empty term range");
        for (int kind = 0; kind < 2; ++kind) {
            const int NL = kind == 0 ? 2 : 4, NW = 1 << NL;
            // this kind's terms [first, last) in its own numbering
            const long base = kind == 0 ? VV : 0, count = kind == 0 ? 2L * L : VV;
            const long first = std::max(0L, r0 - base), last = std::min(count, r1 - base);
            if (last <= first) continue;
            const long nterms = last - first;
            // per-term scratch: all left environments, one site's X / Q / P, two R, G
            long envTot = 0, blk = 0, rmax = 0, gmax = 0;
            std::vector<long> eoff(L + 1);
            for (int s = 0; s <= L; ++s) {
                eoff[s] = envTot;
                envTot += (long)pa[s] * NW * pb[s];
                rmax = std::max(rmax, (long)pa[s] * NW * pb[s]);
            }
            for (int s = 0; s < L; ++s) {
                blk = std::max(blk, (long)pa[s] * NW * 4 * pb[s + 1]);
                gmax = std::max(gmax, (long)pb[s] * 4 * pb[s + 1]);
            }
            const size_t per_term = sizeof(T) * (size_t)(envTot + 3 * blk + 2 * rmax + gmax) +
                                    sizeof(double) * (size_t)(NL * L + 2) + sizeof(T) * (size_t)(NL * L) + 64;
            size_t freeb = 0, totalb = 0;
            THC_CUDA(cudaMemGetInfo(&freeb, &totalb));
            long Bw = batch > 0 ? batch : 4L * E.sms;
            Bw = std::max(1L, std::min<long>({Bw, nterms, (long)(0.4 * freeb / per_term)}));
            Scratch sc(E.al);
            T* Eall = sc.get<T>((size_t)Bw * envTot);
            T* X = sc.get<T>((size_t)Bw * blk);
            T* QY = sc.get<T>((size_t)Bw * blk);
            T* P = sc.get<T>((size_t)Bw * blk);
            T* R[2] = {sc.get<T>((size_t)Bw * rmax), sc.get<T>((size_t)Bw * rmax)};
            T* G = dpsi ? sc.get<T>((size_t)Bw * gmax) : nullptr;
            int* op = sc.get<int>((size_t)Bw * NL);
            T* coef = sc.get<T>((size_t)Bw * NL * L);
            double* weight = sc.get<double>((size_t)Bw);
            double* val = sc.get<double>((size_t)Bw);
            double* g = sc.get<double>((size_t)Bw * NL * L);
            const AdjTerms<T> tm{op, coef, NL, L};
            for (long j0 = 0; j0 < nterms; j0 += Bw) {
                const int Bc = (int)std::min<long>(Bw, nterms - j0);
                const long t0 = first + j0;
                {
                    THC_LAUNCH("adj_terms", st());
                    k_adj_terms<T><<<Bc, 32, 0, st()>>>(kind, t0, Bc, L, N, H->t, H->chi, H->zeta, op, coef, weight);
                }
                E.check();
                THC_CUDA(cudaMemsetAsync(g, 0, sizeof(double) * (size_t)Bc * NL * L, st()));
                {
                    THC_LAUNCH("adj_terms", st());
                    k_adj_boundary<T><<<ceil_div(Bc, 128), 128, 0, st()>>>(Bc, Eall, envTot, R[L & 1], rmax, NW);
                }
                E.check();
                // ---- left sweep: X = E_s psi_s, Y = M_s X, E_{s+1} = phi_s^T Y
                for (int s = 0; s < L; ++s) {
                    const int Da = pa[s], Dap = pa[s + 1], Db = pb[s], Dbp = pb[s + 1];
                    {
                        THC_LAUNCH("adj_gemm", st());
                        E.gemm(Bc, Da * NW, 4 * Dbp, Db, RowMajorA<T>{Eall + eoff[s], envTot, Db},
                               RowMajorB<T>{psi + Bp.off[s], 0, 4 * Dbp}, StoreRM<T>{X, blk, 4 * Dbp});
                    }
                    {
                        THC_LAUNCH("adj_layers", st());
                        dim3 grd(ceil_div(Da * Dbp, 256), Bc);
                        if (NL == 2) k_adj_fwd<T, 2><<<grd, 256, 0, st()>>>(Da, Dbp, blk, X, QY, tm, s);
                        else k_adj_fwd<T, 4><<<grd, 256, 0, st()>>>(Da, Dbp, blk, X, QY, tm, s);
                    }
                    E.check();
                    {
                        THC_LAUNCH("adj_gemm", st());
                        E.gemm(Bc, Dap, NW * Dbp, 4 * Da, AdjTransA<T>{phi + A.off[s], 0, Dap},
                               RowMajorB<T>{QY, blk, NW * Dbp}, StoreRM<T>{Eall + eoff[s + 1], envTot, NW * Dbp});
                    }
                }
                {
                    THC_LAUNCH("adj_terms", st());
                    k_adj_values<T><<<ceil_div(Bc, 128), 128, 0, st()>>>(Bc, Eall + eoff[L], envTot, NW, val);
                }
                E.check();
                // ---- right sweep: Q = phi_s R_{s+1}, P = M_s^T Q (+ coefficient
                // gradients against X = E_s psi_s), R_s = P psi_s^T, G = E_s^T P
                // (skipped when only the value is asked for)
                const bool grads = dt || dchi || dzeta || dpsi;
                for (int s = L - 1; s >= 0 && grads; --s) {
                    const int Da = pa[s], Dap = pa[s + 1], Db = pb[s], Dbp = pb[s + 1];
                    T* Rn = R[(s + 1) & 1];
                    T* Rc = R[s & 1];
                    {
                        THC_LAUNCH("adj_gemm", st());
                        E.gemm(Bc, 4 * Da, NW * Dbp, Dap, RowMajorA<T>{phi + A.off[s], 0, Dap},
                               RowMajorB<T>{Rn, rmax, NW * Dbp}, StoreRM<T>{QY, blk, NW * Dbp});
                    }
                    {
                        THC_LAUNCH("adj_gemm", st());
                        E.gemm(Bc, Da * NW, 4 * Dbp, Db, RowMajorA<T>{Eall + eoff[s], envTot, Db},
                               RowMajorB<T>{psi + Bp.off[s], 0, 4 * Dbp}, StoreRM<T>{X, blk, 4 * Dbp});
                    }
                    {
                        THC_LAUNCH("adj_layers", st());
                        dim3 grd(ceil_div(Da * Dbp, 256), Bc);
                        if (NL == 2) k_adj_bwd<T, 2><<<grd, 256, 0, st()>>>(Da, Dbp, blk, QY, P, X, g, tm, s);
                        else k_adj_bwd<T, 4><<<grd, 256, 0, st()>>>(Da, Dbp, blk, QY, P, X, g, tm, s);
                    }
                    E.check();
                    if (s > 0) {
                        THC_LAUNCH("adj_gemm", st());
                        E.gemm(Bc, Da * NW, Db, 4 * Dbp, RowMajorA<T>{P, blk, 4 * Dbp},
                               TransB<T>{psi + Bp.off[s], 0, 4 * Dbp}, StoreRM<T>{Rc, rmax, Db});
                    }
                    if (dpsi) {
                        {
                            THC_LAUNCH("adj_gemm", st());
                            E.gemm(Bc, Db, 4 * Dbp, Da * NW, AdjTransA<T>{Eall + eoff[s], envTot, Db},
                                   RowMajorB<T>{P, blk, 4 * Dbp}, StoreRM<T>{G, gmax, 4 * Dbp});
                        }
                        const long n = (long)Db * 4 * Dbp;
                        THC_LAUNCH("adj_accum", st());
                        k_adj_accum_site<T><<<std::max(1, (int)std::min<long>(ceil_div((int)std::min<long>(n, 1L << 30), 256), 1024)),
                                              256, 0, st()>>>(Bc, G, gmax, n, weight, dpsi + Bp.off[s]);
                        E.check();
                    }
                }
                {
                    THC_LAUNCH("adj_accum", st());
                    k_adj_params<<<Bc, 32, 0, st()>>>(kind, t0, Bc, L, N, val, g, weight, value_dev, dt, dchi, dzeta);
                }
                E.check();
            }
        }
    }

    // projected problem on the device (float64 single-CTA kernel; the complex
    // Hermitian kernel for complex Krylov vectors).  Outputs: ritz values
    // (mode 0), coefficients of the result on the v_i, the kept rank.
    void krylov_small(int nv, const std::vector<Acc>& Ht, const std::vector<Acc>& S, int mode, double dt,
                      std::vector<double>& ritz, std::vector<c64>& coef, int& rank) {
        if (nv > SMALL_MAX) throw Error(THC_EINVAL, "Krylov dimension above 64");
        Scratch sc(E.al);
        Acc* d = sc.get<Acc>((size_t)2 * nv * nv);
        double* rz = sc.get<double>((size_t)nv);
        c64* cf = sc.get<c64>((size_t)nv);
        int* info = sc.get<int>(2);
        THC_CUDA(cudaMemcpyAsync(d, Ht.data(), nv * nv * sizeof(Acc), cudaMemcpyHostToDevice, st()));
        THC_CUDA(cudaMemcpyAsync(d + nv * nv, S.data(), nv * nv * sizeof(Acc), cudaMemcpyHostToDevice, st()));
        if constexpr (is_complex_v<T>) {
            THC_LAUNCH("krylov_small", st());
            k_krylov_small_c<<<1, 256, KRYLOV_SMEM_C, st()>>>(nv, d, d + nv * nv, mode, dt, 1e-12, rz, cf, info);
        } else {
            double* cr = sc.get<double>((size_t)2 * nv);
            THC_CUDA(cudaMemsetAsync(cr, 0, 2 * nv * sizeof(double), st()));  // mode 0 writes no imaginary part
            {
                THC_LAUNCH("krylov_small", st());
                k_krylov_small<<<1, 256, KRYLOV_SMEM, st()>>>(nv, d, d + nv * nv, mode, dt, 1e-12, rz, cr, cr + nv,
                                                              info);
            }
            E.check();
            {
                THC_LAUNCH("setup", st());
                k_pack_complex<<<1, 64, 0, st()>>>(cf, cr, cr + nv, nv);
            }
        }
        E.check();
        ritz.resize(nv);
        coef.resize(nv);
        int inf[2];
        THC_CUDA(cudaMemcpyAsync(ritz.data(), rz, nv * sizeof(double), cudaMemcpyDeviceToHost, st()));
        THC_CUDA(cudaMemcpyAsync(coef.data(), cf, nv * sizeof(c64), cudaMemcpyDeviceToHost, st()));
        THC_CUDA(cudaMemcpyAsync(inf, info, 2 * sizeof(int), cudaMemcpyDeviceToHost, st()));
        THC_CUDA(cudaStreamSynchronize(st()));
        rank = inf[0];
    }
};

}  // namespace thc
