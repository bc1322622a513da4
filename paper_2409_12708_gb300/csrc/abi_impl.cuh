// abi_impl.cuh -- the typed bodies of the extern "C" entry points (abi.cu),
// one instantiation per storage scalar (float, double, complex float, complex
// double) in its own translation unit (inst_*.cu), so they compile in parallel.
#pragma once

#include <cmath>
#include <string>
#include <type_traits>

#include "engine_ops.cuh"

namespace thc {

void set_last_error(const std::string& msg);  // abi.cu: message for thc_last_error()

namespace abi {

// the float64 accumulator value of a (real or complex) coefficient
template <class Acc>
Acc coef_of(double re, double im) {
    if constexpr (thc::is_complex_v<Acc>) return Acc{re, im};
    else return re;
}

// Shared per-call state: engine, device status word, scratch.
template <class T>
struct Call {
    Engine<T> E;
    Scratch sc;
    Ops<T> ops;
    Call(void* stream, const thc_allocator* a, const thc_opts* o = nullptr)
        : E((cudaStream_t)stream, a), sc(E.al), ops(E) {
        E.tc = o && o->path == THC_PATH_TF32;
        E.dflag = sc.get<int>(1);
        E.ddbg = sc.get<double>(8);
        THC_CUDA(cudaMemsetAsync(E.dflag, 0, sizeof(int), E.st));
        THC_CUDA(cudaMemsetAsync(E.ddbg, 0, 8 * sizeof(double), E.st));
    }
    thc_status finish() {
        int f = 0;
        double d[8];
        THC_CUDA(cudaMemcpyAsync(&f, E.dflag, sizeof(int), cudaMemcpyDeviceToHost, E.st));
        THC_CUDA(cudaMemcpyAsync(d, E.ddbg, 8 * sizeof(double), cudaMemcpyDeviceToHost, E.st));
        THC_CUDA(cudaStreamSynchronize(E.st));
        {
            unsigned long long c[4];
            std::memcpy(c, d + 4, sizeof(c));
            auto& p = thc::profiler();
            std::lock_guard<std::mutex> g(p.mu);
            if (p.on) {  // sweep statistics ride along with the profile
                auto& a = p.acc["jacobi_sweeps_all"];
                a.first += (long)c[1];
                a.second += (double)c[0];
                auto& b = p.acc["jacobi_sweeps_p_ge_128"];
                b.first += (long)c[3];
                b.second += (double)c[2];
            }
        }
        if (f & thc::DEV_NONFINITE) {
            set_last_error("non-finite value met in a decomposition");
            return THC_ENONFINITE;
        }
        if (f & thc::DEV_TC_TIMEOUT) {
            set_last_error("a tensor-core kernel gave up waiting for its MMAs");
            return THC_ETIMEOUT;
        }
        if (f & thc::DEV_SMALL_NONCONV) {
            set_last_error("small eigensolver sweep budget exhausted");
            return THC_ETIMEOUT;
        }
        if (f & thc::DEV_NONCONVERGED) {
            // counted, with the rotations the last sweep still applied: untruncated
            // the projector correction keeps the state exact; truncating, the kept
            // rows are orthogonal only to that sweep's largest rotation
            auto& p = thc::profiler();
            std::lock_guard<std::mutex> g(p.mu);
            auto& x = p.acc["jacobi_budget_exhausted"];
            x.first += 1;
            x.second = std::max(x.second, d[2]);
        }
        return THC_OK;
    }
};

inline std::vector<int> bonds_of(const thc_mps* m) { return std::vector<int>(m->bond, m->bond + m->L + 1); }

inline std::vector<int> pad_up(const std::vector<int>& a, const std::vector<int>& b) {
    std::vector<int> r(a.size());
    for (size_t i = 0; i < a.size(); ++i) r[i] = std::max(a[i], b[i]);
    return r;
}

template <class T>
thc_status apply_H_t(const thc_hamiltonian* H, const thc_mps* psi, const thc_opts* o, thc_mps* out,
                     const thc_allocator* a, void* stream) {
    Call<T> c(stream, a, o);
    const int L = psi->L;
    const auto pf = thc::full_profile(L, o->D_max);
    const auto pin = pad_up(bonds_of(psi), pf);
    T* psi_d = c.sc.template get<T>((size_t)Profile(pin).size);
    c.ops.upload(psi, pin, psi_d);
    T* out_d = c.sc.template get<T>((size_t)Profile(pf).size);
    c.ops.apply_H(H, psi_d, pin, o, out_d);
    c.ops.download(out_d, pf, out, psi->dtype);
    return c.finish();
}

template <class T>
thc_status layer_t(const thc_mps* psi, const double* coef, int sigma, int dagger, const thc_opts* o,
                   thc_mps* out, const thc_allocator* a, void* stream) {
    Call<T> c(stream, a, o);
    c.E.tol_ = o->tol;
    const auto pin = bonds_of(psi);
    T* psi_d = c.sc.template get<T>((size_t)Profile(pin).size);
    c.ops.upload(psi, pin, psi_d);
    thc::Plan P = thc::make_plan<T>(thc::MODE_LAYER, pin, {}, o->D_max);
    T* out_d = c.sc.template get<T>((size_t)Profile(P.out).size);
    std::vector<int> pout;
    c.ops.layer_apply(psi_d, pin, coef, sigma, dagger, o->D_max, out_d, pout, 1);
    c.ops.download(out_d, pout, out, psi->dtype);
    return c.finish();
}

template <class T>
thc_status compress_t(const thc_mps* psi, const thc_opts* o, thc_mps* out, const thc_allocator* a,
                      void* stream) {
    Call<T> c(stream, a, o);
    c.E.tol_ = o->tol;
    const auto pin = bonds_of(psi);
    T* psi_d = c.sc.template get<T>((size_t)Profile(pin).size);
    c.ops.upload(psi, pin, psi_d);
    thc::Plan P = thc::make_plan<T>(thc::MODE_PLAIN, pin, {}, o->D_max);
    T* out_d = c.sc.template get<T>((size_t)Profile(P.out).size);
    std::vector<int> pout;
    c.ops.plain_compress(psi_d, pin, o->D_max, out_d, pout);
    c.ops.download(out_d, pout, out, psi->dtype);
    return c.finish();
}

template <class T>
thc_status inner_t(const thc_mps* phi, const thc_mps* psi, double* re, double* im, void* stream) {
    Call<T> c(stream, nullptr);
    const auto pa = bonds_of(phi), pb = bonds_of(psi);
    T* a = c.sc.template get<T>((size_t)Profile(pa).size);
    T* b = c.sc.template get<T>((size_t)Profile(pb).size);
    c.ops.upload(phi, pa, a);
    c.ops.upload(psi, pb, b);
    const auto v = c.ops.inner1(a, pa, b, pb);
    if constexpr (thc::is_complex_v<T>) {
        *re = v.x;
        if (im) *im = v.y;
    } else {
        *re = v;
        if (im) *im = 0.0;
    }
    return c.finish();
}

template <class T>
thc_status add_t(int n, const double* cre, const double* cim, const thc_mps* const* xs, const thc_opts* o,
                 thc_mps* out, const thc_allocator* a, void* stream) {
    using Acc = typename thc::Wide<T>::type;
    Call<T> c(stream, a, o);
    c.E.tol_ = o->tol;
    const int L = xs[0]->L;
    const auto pf = thc::full_profile(L, o->D_max);
    const long sz = Profile(pf).size;
    T* buf = c.sc.template get<T>((size_t)n * sz);
    std::vector<const T*> ptrs(n);
    for (int i = 0; i < n; ++i) {
        for (int b = 0; b <= L; ++b)
            if (xs[i]->bond[b] > pf[b])
                throw Error(THC_EUNSUPPORTED, "add_compress inputs must have bonds <= min(D_max, 4^b, 4^(L-b))");
        c.ops.upload(xs[i], pf, buf + (long)i * sz);
        ptrs[i] = buf + (long)i * sz;
    }
    std::vector<Acc> cs(n);
    for (int i = 0; i < n; ++i) cs[i] = coef_of<Acc>(cre[i], cim ? cim[i] : 0.0);
    T* out_d = c.sc.template get<T>((size_t)sz);
    c.ops.add_compress(n, cs.data(), ptrs.data(), pf, o->D_max, out_d);
    c.ops.download(out_d, pf, out, xs[0]->dtype);
    return c.finish();
}

template <class T>
thc_status lanczos_t(const thc_hamiltonian* H, const thc_mps* psi0, int K, const thc_opts* o,
                     double* energy, double* ritz, thc_mps* ground, const thc_allocator* a, void* stream) {
    Call<T> c(stream, a, o);
    const int L = psi0->L;
    const auto pf = thc::full_profile(L, o->D_max);
    for (int b = 0; b <= L; ++b)
        if (psi0->bond[b] > pf[b])
            throw Error(THC_EUNSUPPORTED, "psi0 bonds must be <= min(D_max, 4^b, 4^(L-b))");
    const long sz = Profile(pf).size;
    T* p0 = c.sc.template get<T>((size_t)sz);
    c.ops.upload(psi0, pf, p0);
    T* vbuf = c.sc.template get<T>((size_t)K * sz);
    T* wbuf = c.sc.template get<T>((size_t)K * sz);
    using Acc = typename thc::Wide<T>::type;
    std::vector<Acc> Ht, S;
    std::vector<double> rz;
    std::vector<c64> cf;
    const int nv = c.ops.krylov_basis(H, p0, pf, K, o, vbuf, wbuf, Ht, S);
    int rank = 0;
    c.ops.krylov_small(nv, Ht, S, 0, 0.0, rz, cf, rank);
    if (rank < 1) throw Error(THC_EBREAKDOWN, "no Krylov vector survived canonical orthogonalisation");
    *energy = rz[0];
    if (ritz)
        for (int i = 0; i < K; ++i) ritz[i] = i < rank ? rz[i] : std::nan("");
    if (ground) {
        std::vector<const T*> xs(nv);
        std::vector<Acc> cs(nv);
        for (int i = 0; i < nv; ++i) {
            xs[i] = vbuf + (long)i * sz;
            cs[i] = coef_of<Acc>(cf[i].x, cf[i].y);
        }
        T* g = c.sc.template get<T>((size_t)sz);
        c.ops.add_compress(nv, cs.data(), xs.data(), pf, o->D_max, g);
        c.ops.download(g, pf, ground, psi0->dtype);
    }
    return c.finish();
}

// Restarted Lanczos (Sec. 2.2): `cycles` runs of K-step Lanczos, each started
// from the previous run's lowest Ritz vector sum_i (C y_0)_i v_i (pairwise
// reduction, normalised); with lower states every run is kept orthogonal to
// them (excited states).  energies[c] = lowest Ritz value of run c; state:
// optional output, the last Ritz vector.
template <class T>
thc_status restarted_t(const thc_hamiltonian* H, const thc_mps* psi0, int K, int cycles, int n_lower,
                       const thc_mps* const* lower, const thc_opts* o, double* energies, thc_mps* state,
                       const thc_allocator* a, void* stream) {
    using Acc = typename thc::Wide<T>::type;
    Call<T> c(stream, a, o);
    const int L = psi0->L;
    const auto pf = thc::full_profile(L, o->D_max);
    auto check_bonds = [&](const thc_mps* m) {
        for (int b = 0; b <= L; ++b)
            if (m->bond[b] > pf[b])
                throw Error(THC_EUNSUPPORTED, "MPS bonds must be <= min(D_max, 4^b, 4^(L-b))");
    };
    check_bonds(psi0);
    const long sz = Profile(pf).size;
    std::vector<const T*> low(n_lower);
    for (int m = 0; m < n_lower; ++m) {
        check_bonds(lower[m]);
        T* d = c.sc.template get<T>((size_t)sz);
        c.ops.upload(lower[m], pf, d);
        low[m] = d;
    }
    T* x = c.sc.template get<T>((size_t)sz);
    c.ops.upload(psi0, pf, x);
    T* vbuf = c.sc.template get<T>((size_t)K * sz);
    T* wbuf = c.sc.template get<T>((size_t)K * sz);
    for (int cy = 0; cy < cycles; ++cy) {
        std::vector<Acc> Ht, S;
        std::vector<double> rz;
        std::vector<c64> cf;
        const int nv = c.ops.krylov_basis(H, x, pf, K, o, vbuf, wbuf, Ht, S, low);
        int rank = 0;
        c.ops.krylov_small(nv, Ht, S, 0, 0.0, rz, cf, rank);
        if (rank < 1) throw Error(THC_EBREAKDOWN, "no Krylov vector survived canonical orthogonalisation");
        energies[cy] = rz[0];
        std::vector<const T*> xs(nv);
        std::vector<Acc> cs(nv);
        for (int i = 0; i < nv; ++i) {
            xs[i] = vbuf + (long)i * sz;
            cs[i] = coef_of<Acc>(cf[i].x, cf[i].y);
        }
        c.ops.add_compress(nv, cs.data(), xs.data(), pf, o->D_max, x);
        const double nx = std::sqrt(std::fabs(thc::treal_part(c.ops.inner1(x, pf, x, pf))));
        if (!(nx > 0.0)) throw Error(THC_EBREAKDOWN, "vanishing Ritz vector");
        const Profile P(pf);
        THC_LAUNCH("scale", c.E.st);
        thc::k_scale<T><<<64, 256, 0, c.E.st>>>(x + P.off[L - 1], P.site_size(L - 1), coef_of<Acc>(1.0 / nx, 0.0));
        c.E.check();
    }
    if (state) c.ops.download(x, pf, state, psi0->dtype);
    return c.finish();
}

// Exact <phi|H|psi> and its derivatives (the adjoint): real MPS of the path's
// precision.  grad_t / grad_chi / grad_zeta: device float64 arrays (written;
// may be null); grad_psi: optional output MPS with psi's bonds and dtype.
template <class T>
thc_status expect_grad_t(const thc_hamiltonian* H, const thc_mps* phi, const thc_mps* psi, const thc_opts* o,
                         double* value, double* grad_t, double* grad_chi, double* grad_zeta, thc_mps* grad_psi,
                         const thc_allocator* a, void* stream) {
    Call<T> c(stream, a, o);
    const int L = psi->L, N = H->N;
    const auto pa = bonds_of(phi), pb = bonds_of(psi);
    T* pd = c.sc.template get<T>((size_t)Profile(pa).size);
    T* qd = c.sc.template get<T>((size_t)Profile(pb).size);
    c.ops.upload(phi, pa, pd);
    c.ops.upload(psi, pb, qd);
    double* vd = c.sc.template get<double>(1);
    THC_CUDA(cudaMemsetAsync(vd, 0, sizeof(double), c.E.st));
    if (grad_t) THC_CUDA(cudaMemsetAsync(grad_t, 0, sizeof(double) * L * L, c.E.st));
    if (grad_chi) THC_CUDA(cudaMemsetAsync(grad_chi, 0, sizeof(double) * L * N, c.E.st));
    if (grad_zeta) THC_CUDA(cudaMemsetAsync(grad_zeta, 0, sizeof(double) * N * N, c.E.st));
    T* gd = nullptr;
    if (grad_psi) {
        gd = c.sc.template get<T>((size_t)Profile(pb).size);
        THC_CUDA(cudaMemsetAsync(gd, 0, sizeof(T) * Profile(pb).size, c.E.st));
    }
    c.ops.expect_grad(H, pd, pa, qd, pb, o->batch, o->term_begin, o->term_end, vd, grad_t, grad_chi, grad_zeta, gd);
    THC_CUDA(cudaMemcpyAsync(value, vd, sizeof(double), cudaMemcpyDeviceToHost, c.E.st));
    if (grad_psi) c.ops.download(gd, pb, grad_psi, psi->dtype);
    return c.finish();
}

// One global-Krylov time step (Sec. 2.2, Eq. Krylov_combination) on complex
// site tensors T: K vectors from psi/|psi|, the projected problem with
// a(dt) = exp(-i dt Heff) a(0) in the orthonormalised basis, the combination
// sum_i (|psi| a_i) v_i by the pairwise reduction, renormalised to |psi|.
template <class T>
thc_status expm_t(const thc_hamiltonian* H, const thc_mps* psi, double dt, int K, const thc_opts* o, thc_mps* out,
                  double* lost_norm, const thc_allocator* a, void* stream) {
    static_assert(thc::is_complex_v<T>, "time evolution runs on complex tensors");
    Call<T> c(stream, a, o);
    const int L = psi->L;
    const auto pf = thc::full_profile(L, o->D_max);
    for (int b = 0; b <= L; ++b)
        if (psi->bond[b] > pf[b])
            throw Error(THC_EUNSUPPORTED, "psi bonds must be <= min(D_max, 4^b, 4^(L-b))");
    const long sz = Profile(pf).size;
    T* p0 = c.sc.template get<T>((size_t)sz);
    c.ops.upload(psi, pf, p0);
    const double n0 = std::sqrt(std::fabs(c.ops.inner1(p0, pf, p0, pf).x));
    if (!(n0 > 0.0)) throw Error(THC_EBREAKDOWN, "zero initial state");
    T* vbuf = c.sc.template get<T>((size_t)K * sz);
    T* wbuf = c.sc.template get<T>((size_t)K * sz);
    std::vector<c64> Ht, S, cf;
    std::vector<double> rz;
    const int nv = c.ops.krylov_basis(H, p0, pf, K, o, vbuf, wbuf, Ht, S);
    int rank = 0;
    c.ops.krylov_small(nv, Ht, S, 1, dt, rz, cf, rank);
    if (rank < 1) throw Error(THC_EBREAKDOWN, "no Krylov vector survived canonical orthogonalisation");
    std::vector<const T*> xs(nv);
    std::vector<c64> cs(nv);
    for (int i = 0; i < nv; ++i) {
        xs[i] = vbuf + (long)i * sz;
        cs[i] = c64{cf[i].x * n0, cf[i].y * n0};
    }
    T* r = c.sc.template get<T>((size_t)sz);
    c.ops.add_compress(nv, cs.data(), xs.data(), pf, o->D_max, r);
    const double n1 = std::sqrt(std::fabs(c.ops.inner1(r, pf, r, pf).x));
    if (!(n1 > 0.0)) throw Error(THC_EBREAKDOWN, "the time-evolved state vanished");
    if (lost_norm) *lost_norm = std::max(0.0, 1.0 - n1 / n0);
    {
        const Profile P(pf);
        THC_LAUNCH("scale", c.E.st);
        thc::k_scale<T><<<64, 256, 0, c.E.st>>>(r + P.off[L - 1], P.site_size(L - 1), c64{n0 / n1, 0.0});
    }
    c.E.check();
    c.ops.download(r, pf, out, std::is_same<T, c64>::value ? THC_C128 : THC_C64);
    return c.finish();
}

}  // namespace abi
}  // namespace thc

// Explicit instantiations: THC_ABI_INSTANTIATE(T) in the inst_*.cu files,
// declared extern in abi.cu.
#define THC_ABI_FOR(PREFIX, T)                                                                                  \
    PREFIX thc_status thc::abi::apply_H_t<T>(const thc_hamiltonian*, const thc_mps*, const thc_opts*, thc_mps*,  \
                                             const thc_allocator*, void*);                                      \
    PREFIX thc_status thc::abi::layer_t<T>(const thc_mps*, const double*, int, int, const thc_opts*, thc_mps*,    \
                                           const thc_allocator*, void*);                                        \
    PREFIX thc_status thc::abi::compress_t<T>(const thc_mps*, const thc_opts*, thc_mps*, const thc_allocator*,   \
                                              void*);                                                           \
    PREFIX thc_status thc::abi::inner_t<T>(const thc_mps*, const thc_mps*, double*, double*, void*);           \
    PREFIX thc_status thc::abi::add_t<T>(int, const double*, const double*, const thc_mps* const*,              \
                                         const thc_opts*, thc_mps*, const thc_allocator*, void*);               \
    PREFIX thc_status thc::abi::lanczos_t<T>(const thc_hamiltonian*, const thc_mps*, int, const thc_opts*,      \
                                             double*, double*, thc_mps*, const thc_allocator*, void*);         \
    PREFIX thc_status thc::abi::restarted_t<T>(const thc_hamiltonian*, const thc_mps*, int, int, int,           \
                                               const thc_mps* const*, const thc_opts*, double*, thc_mps*,        \
                                               const thc_allocator*, void*);
#define THC_ABI_FOR_REAL(PREFIX, T)                                                                             \
    PREFIX thc_status thc::abi::expect_grad_t<T>(const thc_hamiltonian*, const thc_mps*, const thc_mps*,         \
                                                 const thc_opts*, double*, double*, double*, double*, thc_mps*,  \
                                                 const thc_allocator*, void*);
#define THC_ABI_FOR_EXPM(PREFIX, T)                                                                             \
    PREFIX thc_status thc::abi::expm_t<T>(const thc_hamiltonian*, const thc_mps*, double, int, const thc_opts*,  \
                                          thc_mps*, double*, const thc_allocator*, void*);
