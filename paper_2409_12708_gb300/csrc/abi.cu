// abi.cu -- extern "C" entry points declared in include/thc.h.
#include <cmath>
#include <string>

#include "engine_ops.cuh"

#define THC_STR2(x) #x
#define THC_STR(x) THC_STR2(x)

using thc::Engine;
using thc::Error;
using thc::Ops;
using thc::Profile;
using thc::Scratch;

namespace {

thread_local std::string g_err;

thc_status fail(thc_status s, const std::string& m) {
    g_err = m;
    return s;
}

size_t dtype_size(thc_dtype d) {
    switch (d) {
        case THC_F64: return 8;
        case THC_F32: return 4;
        case THC_C64: return 8;
        case THC_C128: return 16;
    }
    return 0;
}

void check_mps(const thc_mps* m, const char* what) {
    if (!m) throw Error(THC_EINVAL, std::string(what) + ": null descriptor");
    if (m->L < 2 || m->L > THC_MAX_SITES)
        throw Error(THC_EINVAL, std::string(what) + ": L must be in [2, " + std::to_string(THC_MAX_SITES) + "]");
    if (m->d != 4) throw Error(THC_EINVAL, std::string(what) + ": d must be 4");
    if (m->bond[0] != 1 || m->bond[m->L] != 1)
        throw Error(THC_EINVAL, std::string(what) + ": boundary bonds must be 1");
    for (int b = 0; b <= m->L; ++b)
        if (m->bond[b] < 1 || m->bond[b] > 4096) throw Error(THC_EINVAL, std::string(what) + ": bad bond");
    for (int s = 0; s < m->L; ++s)
        if (!m->site[s]) throw Error(THC_EINVAL, std::string(what) + ": null site pointer");
    if (dtype_size(m->dtype) == 0) throw Error(THC_EINVAL, std::string(what) + ": bad dtype");
}

void check_opts(const thc_opts* o) {
    if (!o) throw Error(THC_EINVAL, "null options");
    if (o->D_max < 1) throw Error(THC_EINVAL, "D_max must be >= 1");
    if (!(o->tol >= 0.0) || o->tol >= 1.0) throw Error(THC_EINVAL, "tol must be in [0, 1)");
    if (o->path != THC_PATH_FP64 && o->path != THC_PATH_FP32) throw Error(THC_EINVAL, "bad path");
    if (o->D_max > 512) throw Error(THC_EUNSUPPORTED, "D_max above 512 is not supported");
}

void check_ham(const thc_hamiltonian* H, int L) {
    if (!H || !H->t || !H->chi || !H->zeta) throw Error(THC_EINVAL, "null Hamiltonian array");
    if (H->L != L) throw Error(THC_EINVAL, "Hamiltonian L differs from the MPS");
    if (H->N < 1 || H->N > 4096) throw Error(THC_EINVAL, "THC rank N out of range");
}

thc_dtype real_dtype(thc_path p) { return p == THC_PATH_FP64 ? THC_F64 : THC_F32; }

void check_path_dtype(const thc_mps* m, const thc_opts* o) {
    if (m->dtype != real_dtype(o->path))
        throw Error(THC_EINVAL, "MPS dtype does not match the compute path (F64 for FP64, F32 for FP32)");
}

// Shared per-call state: engine, device status word, scratch.
template <class T>
struct Call {
    Engine<T> E;
    Scratch sc;
    Ops<T> ops;
    Call(void* stream, const thc_allocator* a)
        : E((cudaStream_t)stream, a), sc(E.al), ops(E) {
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
        if (f & thc::DEV_NONFINITE) return fail(THC_ENONFINITE, "non-finite value met in a decomposition");
        if (f & thc::DEV_SMALL_NONCONV) return fail(THC_ETIMEOUT, "small eigensolver sweep budget exhausted");
        if (f & thc::DEV_NONCONVERGED) {
            // not an error: the projector correction keeps the state exact and the
            // kept subspace is orthogonal to the rotation threshold of the last
            // sweep; counted, with the rotations that sweep still applied
            auto& p = thc::profiler();
            std::lock_guard<std::mutex> g(p.mu);
            auto& x = p.acc["jacobi_budget_exhausted"];
            x.first += 1;
            x.second = std::max(x.second, d[2]);
        }
        return THC_OK;
    }
};

std::vector<int> bonds_of(const thc_mps* m) { return std::vector<int>(m->bond, m->bond + m->L + 1); }

std::vector<int> pad_up(const std::vector<int>& a, const std::vector<int>& b) {
    std::vector<int> r(a.size());
    for (size_t i = 0; i < a.size(); ++i) r[i] = std::max(a[i], b[i]);
    return r;
}

template <class T>
thc_status apply_H_t(const thc_hamiltonian* H, const thc_mps* psi, const thc_opts* o, thc_mps* out,
                     const thc_allocator* a, void* stream) {
    Call<T> c(stream, a);
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
    Call<T> c(stream, a);
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
    Call<T> c(stream, a);
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
thc_status inner_t(const thc_mps* phi, const thc_mps* psi, double* re, void* stream) {
    Call<T> c(stream, nullptr);
    const auto pa = bonds_of(phi), pb = bonds_of(psi);
    T* a = c.sc.template get<T>((size_t)Profile(pa).size);
    T* b = c.sc.template get<T>((size_t)Profile(pb).size);
    c.ops.upload(phi, pa, a);
    c.ops.upload(psi, pb, b);
    *re = c.ops.inner1(a, pa, b, pb);
    return c.finish();
}

template <class T>
thc_status add_t(int n, const double* cre, const thc_mps* const* xs, const thc_opts* o, thc_mps* out,
                 const thc_allocator* a, void* stream) {
    Call<T> c(stream, a);
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
    T* out_d = c.sc.template get<T>((size_t)sz);
    c.ops.add_compress(n, cre, ptrs.data(), pf, o->D_max, out_d);
    c.ops.download(out_d, pf, out, xs[0]->dtype);
    return c.finish();
}

template <class T>
thc_status lanczos_t(const thc_hamiltonian* H, const thc_mps* psi0, int K, const thc_opts* o,
                     double* energy, double* ritz, thc_mps* ground, const thc_allocator* a, void* stream) {
    Call<T> c(stream, a);
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
    std::vector<double> Ht, S, rz, cre, cim;
    const int nv = c.ops.krylov_basis(H, p0, pf, K, o, vbuf, wbuf, Ht, S);
    int rank = 0;
    c.ops.krylov_small(nv, Ht, S, 0, 0.0, rz, cre, cim, rank);
    if (rank < 1) throw Error(THC_EBREAKDOWN, "no Krylov vector survived canonical orthogonalisation");
    *energy = rz[0];
    if (ritz)
        for (int i = 0; i < K; ++i) ritz[i] = i < rank ? rz[i] : std::nan("");
    if (ground) {
        std::vector<const T*> xs(nv);
        for (int i = 0; i < nv; ++i) xs[i] = vbuf + (long)i * sz;
        T* g = c.sc.template get<T>((size_t)sz);
        c.ops.add_compress(nv, cre.data(), xs.data(), pf, o->D_max, g);
        c.ops.download(g, pf, ground, psi0->dtype);
    }
    return c.finish();
}

#define THC_GUARD(...)                                                    \
    try {                                                                 \
        __VA_ARGS__                                                       \
    } catch (const Error& e) {                                            \
        return fail(e.st, e.what());                                      \
    } catch (const std::exception& e) {                                   \
        return fail(THC_ECUDA, e.what());                                 \
    }

}  // namespace

namespace thc {
// lets other translation units report through thc_last_error()
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace thc

extern "C" {

thc_status thc_apply_H(const thc_hamiltonian* H, const thc_mps* psi, const thc_opts* opts, thc_mps* out,
                       const thc_allocator* alloc, void* stream) {
    THC_GUARD({
        check_mps(psi, "psi");
        check_opts(opts);
        check_ham(H, psi->L);
        check_path_dtype(psi, opts);
        if (!out) throw Error(THC_EINVAL, "null output");
        if (opts->path == THC_PATH_FP64) return apply_H_t<double>(H, psi, opts, out, alloc, stream);
        return apply_H_t<float>(H, psi, opts, out, alloc, stream);
    })
}

thc_status thc_layer_apply(const thc_mps* psi, const double* coef, int sigma, int dagger,
                           const thc_opts* opts, thc_mps* out, const thc_allocator* alloc, void* stream) {
    THC_GUARD({
        check_mps(psi, "psi");
        check_opts(opts);
        check_path_dtype(psi, opts);
        if (!coef || !out) throw Error(THC_EINVAL, "null coefficient or output");
        if (sigma != 0 && sigma != 1) throw Error(THC_EINVAL, "sigma must be 0 or 1");
        if (opts->path == THC_PATH_FP64) return layer_t<double>(psi, coef, sigma, dagger, opts, out, alloc, stream);
        return layer_t<float>(psi, coef, sigma, dagger, opts, out, alloc, stream);
    })
}

thc_status thc_compress(const thc_mps* psi, const thc_opts* opts, thc_mps* out,
                        const thc_allocator* alloc, void* stream) {
    THC_GUARD({
        check_mps(psi, "psi");
        check_opts(opts);
        check_path_dtype(psi, opts);
        if (!out) throw Error(THC_EINVAL, "null output");
        if (opts->path == THC_PATH_FP64) return compress_t<double>(psi, opts, out, alloc, stream);
        return compress_t<float>(psi, opts, out, alloc, stream);
    })
}

thc_status mps_inner(const thc_mps* phi, const thc_mps* psi, double* out_re, double* out_im, void* stream) {
    THC_GUARD({
        check_mps(phi, "phi");
        check_mps(psi, "psi");
        if (phi->L != psi->L) throw Error(THC_EINVAL, "L mismatch");
        if (phi->dtype != psi->dtype) throw Error(THC_EINVAL, "dtype mismatch");
        if (!out_re) throw Error(THC_EINVAL, "null output");
        if (out_im) *out_im = 0.0;
        if (phi->dtype == THC_F64) return inner_t<double>(phi, psi, out_re, stream);
        if (phi->dtype == THC_F32) return inner_t<float>(phi, psi, out_re, stream);
        throw Error(THC_EUNSUPPORTED, "complex MPS are not supported by this build");
    })
}

thc_status mps_add_compress(int n, const double* coeff_re, const double* coeff_im, const thc_mps* const* xs,
                            const thc_opts* opts, thc_mps* out, const thc_allocator* alloc, void* stream) {
    THC_GUARD({
        if (n < 1 || !xs || !coeff_re || !out) throw Error(THC_EINVAL, "bad add_compress arguments");
        check_opts(opts);
        for (int i = 0; i < n; ++i) {
            check_mps(xs[i], "x");
            check_path_dtype(xs[i], opts);
            if (xs[i]->L != xs[0]->L) throw Error(THC_EINVAL, "L mismatch");
        }
        if (coeff_im)
            for (int i = 0; i < n; ++i)
                if (coeff_im[i] != 0.0) throw Error(THC_EUNSUPPORTED, "complex coefficients are not supported");
        if (opts->path == THC_PATH_FP64) return add_t<double>(n, coeff_re, xs, opts, out, alloc, stream);
        return add_t<float>(n, coeff_re, xs, opts, out, alloc, stream);
    })
}

thc_status krylov_lanczos_ground(const thc_hamiltonian* H, const thc_mps* psi0, int K, const thc_opts* opts,
                                 double* energy, double* ritz, thc_mps* ground,
                                 const thc_allocator* alloc, void* stream) {
    THC_GUARD({
        check_mps(psi0, "psi0");
        check_opts(opts);
        check_ham(H, psi0->L);
        check_path_dtype(psi0, opts);
        if (K < 1 || K > thc::SMALL_MAX) throw Error(THC_EINVAL, "K must be in [1, 64]");
        if (!energy) throw Error(THC_EINVAL, "null energy");
        if (opts->path == THC_PATH_FP64)
            return lanczos_t<double>(H, psi0, K, opts, energy, ritz, ground, alloc, stream);
        return lanczos_t<float>(H, psi0, K, opts, energy, ritz, ground, alloc, stream);
    })
}

thc_status krylov_expm_apply(const thc_hamiltonian* H, const thc_mps* psi, double dt, int K,
                             const thc_opts* opts, thc_mps* out, double* lost_norm,
                             const thc_allocator* alloc, void* stream) {
    (void)H; (void)psi; (void)dt; (void)K; (void)opts; (void)out; (void)lost_norm; (void)alloc; (void)stream;
    return fail(THC_EUNSUPPORTED, "complex MPS (time evolution) are not supported by this build");
}

thc_status thc_kinetic_factors(int L, const double* t, double* lambda, double* u, void* stream) {
    THC_GUARD({
        if (L < 1 || L > thc::SMALL_MAX || !t || !lambda || !u) throw Error(THC_EINVAL, "bad arguments");
        Engine<double> E((cudaStream_t)stream, nullptr);
        Scratch sc(E.al);
        int* flag = sc.get<int>(1);
        THC_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), E.st));
        thc::k_kinetic_factors<<<1, 256, thc::KINETIC_SMEM, E.st>>>(L, t, lambda, u, flag);
        E.check();
        int f = 0;
        THC_CUDA(cudaMemcpyAsync(&f, flag, sizeof(int), cudaMemcpyDeviceToHost, E.st));
        THC_CUDA(cudaStreamSynchronize(E.st));
        if (f) return fail(THC_ETIMEOUT, "Jacobi sweep budget exhausted");
        return THC_OK;
    })
}

void thc_mps_free(thc_mps* m, const thc_allocator* alloc, void* stream) {
    if (!m || !m->owner) return;
    thc::Alloc al;
    al.a = alloc;
    al.st = (cudaStream_t)stream;
    al.put(m->owner);
    std::memset(m, 0, sizeof(*m));
}

const char* thc_last_error(void) { return g_err.c_str(); }

unsigned long long thc_kernel_launches(void) { return thc::profiler().launches.load(); }

void thc_profile_enable(int on) {
    auto& p = thc::profiler();
    std::lock_guard<std::mutex> g(p.mu);
    p.on = on != 0;
}

int thc_profile_read(char* buf, int len) {
    auto& p = thc::profiler();
    std::string js = "{";
    {
        std::lock_guard<std::mutex> g(p.mu);
        p.drain();
        bool first = true;
        for (auto& kv : p.acc) {
            char tmp[256];
            snprintf(tmp, sizeof(tmp), "%s\"%s\": {\"launches\": %ld, \"ms\": %.6f}", first ? "" : ", ",
                     kv.first.c_str(), kv.second.first, kv.second.second);
            js += tmp;
            first = false;
        }
        p.acc.clear();
    }
    js += "}";
    if (buf && len > 0) {
        const int n = std::min<int>(len - 1, (int)js.size());
        std::memcpy(buf, js.data(), n);
        buf[n] = 0;
    }
    return (int)js.size() + 1;
}

const char* thc_build_info(void) {
    return "thc-mpo gb300: sm_103a, CUDA " THC_STR(__CUDACC_VER_MAJOR__) "." THC_STR(__CUDACC_VER_MINOR__);
}

}  // extern "C"
