// abi.cu -- extern "C" entry points declared in include/thc.h.
#include <cmath>
#include <string>
#include <thread>
#include <type_traits>

#include "abi_impl.cuh"

#define THC_STR2(x) #x
#define THC_STR(x) THC_STR2(x)

using thc::c32;
using thc::c64;
using thc::Error;
using thc::Scratch;
using namespace thc::abi;

// the typed bodies are compiled in inst_*.cu
THC_ABI_FOR(extern template, double)
THC_ABI_FOR(extern template, float)
THC_ABI_FOR(extern template, c64)
THC_ABI_FOR(extern template, c32)
THC_ABI_FOR_EXPM(extern template, c64)
THC_ABI_FOR_EXPM(extern template, c32)
THC_ABI_FOR_REAL(extern template, double)
THC_ABI_FOR_REAL(extern template, float)

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
    if (o->path != THC_PATH_FP64 && o->path != THC_PATH_FP32 && o->path != THC_PATH_TF32)
        throw Error(THC_EINVAL, "bad path");
    if (o->D_max > 512) throw Error(THC_EUNSUPPORTED, "D_max above 512 is not supported");
    if (o->merge_spin != 0 && o->merge_spin != 1) throw Error(THC_EINVAL, "merge_spin must be 0 or 1");
}

void check_ham(const thc_hamiltonian* H, int L) {
    if (!H || !H->t || !H->chi || !H->zeta) throw Error(THC_EINVAL, "null Hamiltonian array");
    if (H->L != L) throw Error(THC_EINVAL, "Hamiltonian L differs from the MPS");
    if (H->N < 1 || H->N > 4096) throw Error(THC_EINVAL, "THC rank N out of range");
}

thc_dtype real_dtype(thc_path p) { return p == THC_PATH_FP64 ? THC_F64 : THC_F32; }
thc_dtype complex_dtype(thc_path p) { return p == THC_PATH_FP64 ? THC_C128 : THC_C64; }  // FP32, TF32: C64
bool is_complex(thc_dtype d) { return d == THC_C64 || d == THC_C128; }

void check_path_dtype(const thc_mps* m, const thc_opts* o) {
    if (m->dtype != real_dtype(o->path) && m->dtype != complex_dtype(o->path))
        throw Error(THC_EINVAL, "MPS dtype does not match the compute path (F64 or C128 for FP64, F32 or C64 "
                                "for FP32 and TF32)");
}

// Call f with a null pointer of the storage scalar of dtype d (the engine's T).
template <class F>
thc_status dispatch(thc_dtype d, F&& f) {
    switch (d) {
        case THC_F64: return f((double*)nullptr);
        case THC_F32: return f((float*)nullptr);
        case THC_C128: return f((c64*)nullptr);
        case THC_C64: return f((c32*)nullptr);
    }
    throw Error(THC_EINVAL, "bad dtype");
}

// complex MPS support the bond dimensions of D_max <= 256
void check_complex_dmax(thc_dtype d, const thc_opts* o) {
    if (is_complex(d) && o->D_max > 256) throw Error(THC_EUNSUPPORTED, "complex MPS: D_max above 256 is not supported");
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
        check_complex_dmax(psi->dtype, opts);
        if (!out) throw Error(THC_EINVAL, "null output");
        return dispatch(psi->dtype, [&](auto* tag) {
            using T = std::remove_pointer_t<decltype(tag)>;
            return apply_H_t<T>(H, psi, opts, out, alloc, stream);
        });
    })
}

thc_status thc_apply_H_batched(int n, const thc_hamiltonian* const* H, const thc_mps* const* psi,
                               const thc_opts* opts, thc_mps* out, const thc_allocator* alloc, void* stream) {
    THC_GUARD({
        if (n < 1 || !H || !psi || !out) throw Error(THC_EINVAL, "bad batched arguments");
        check_opts(opts);
        for (int i = 0; i < n; ++i) {
            check_mps(psi[i], "psi");
            check_ham(H[i], psi[i]->L);
            check_path_dtype(psi[i], opts);
            check_complex_dmax(psi[i]->dtype, opts);
            if (psi[i]->dtype != psi[0]->dtype) throw Error(THC_EINVAL, "all instances share one dtype");
        }
        for (int i = 0; i < n; ++i) std::memset(&out[i], 0, sizeof(thc_mps));
        // the instances' terms in flight share the device: split the default
        thc_opts o = *opts;
        if (o.batch <= 0) {
            int dev = 0, sms = 152;
            THC_CUDA(cudaGetDevice(&dev));
            THC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            o.batch = std::max(32, 4 * sms / n);
        }
        const cudaStream_t parent = (cudaStream_t)stream;
        int cur_dev = 0;
        THC_CUDA(cudaGetDevice(&cur_dev));  // worker threads start on device 0: they take the caller's
        cudaEvent_t fork;
        THC_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        THC_CUDA(cudaEventRecord(fork, parent));
        std::vector<cudaStream_t> st(n, nullptr);
        std::vector<cudaEvent_t> join(n, nullptr);
        std::vector<thc_status> status(n, THC_OK);
        std::vector<std::string> msg(n);
        thc_status setup = THC_OK;
        for (int i = 0; i < n && setup == THC_OK; ++i) {
            if (cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaStreamWaitEvent(st[i], fork, 0) != cudaSuccess)
                setup = THC_ECUDA;
        }
        if (setup == THC_OK) {
            // one host thread per instance: each drives its own engine on its own stream
            std::vector<std::thread> th;
            for (int i = 0; i < n; ++i)
                th.emplace_back([&, i] {
                    if (cudaSetDevice(cur_dev) != cudaSuccess) {
                        status[i] = THC_ECUDA;
                        msg[i] = "cudaSetDevice failed in the instance's thread";
                        return;
                    }
                    status[i] = thc_apply_H(H[i], psi[i], &o, &out[i], alloc, (void*)st[i]);
                    if (status[i] != THC_OK) msg[i] = thc_last_error();
                });
            for (auto& t : th) t.join();
        }
        for (int i = 0; i < n; ++i) {
            if (st[i] && join[i]) {
                cudaEventRecord(join[i], st[i]);
                cudaStreamWaitEvent(parent, join[i], 0);
            }
        }
        for (int i = 0; i < n; ++i) {
            if (join[i]) cudaEventDestroy(join[i]);
            if (st[i]) cudaStreamDestroy(st[i]);
        }
        cudaEventDestroy(fork);
        if (setup != THC_OK) throw Error(THC_ECUDA, "could not create the instances' streams");
        for (int i = 0; i < n; ++i)
            if (status[i] != THC_OK) {
                // release what the other instances returned; report the first failure
                for (int j = 0; j < n; ++j) thc_mps_free(&out[j], alloc, stream);
                return fail(status[i], "instance " + std::to_string(i) + ": " + msg[i]);
            }
        return THC_OK;
    })
}

thc_status thc_layer_apply(const thc_mps* psi, const double* coef, int sigma, int dagger,
                           const thc_opts* opts, thc_mps* out, const thc_allocator* alloc, void* stream) {
    THC_GUARD({
        check_mps(psi, "psi");
        check_opts(opts);
        check_path_dtype(psi, opts);
        check_complex_dmax(psi->dtype, opts);
        if (!coef || !out) throw Error(THC_EINVAL, "null coefficient or output");
        if (sigma != 0 && sigma != 1) throw Error(THC_EINVAL, "sigma must be 0 or 1");
        return dispatch(psi->dtype, [&](auto* tag) {
            using T = std::remove_pointer_t<decltype(tag)>;
            return layer_t<T>(psi, coef, sigma, dagger, opts, out, alloc, stream);
        });
    })
}

thc_status thc_compress(const thc_mps* psi, const thc_opts* opts, thc_mps* out,
                        const thc_allocator* alloc, void* stream) {
    THC_GUARD({
        check_mps(psi, "psi");
        check_opts(opts);
        check_path_dtype(psi, opts);
        check_complex_dmax(psi->dtype, opts);
        if (!out) throw Error(THC_EINVAL, "null output");
        return dispatch(psi->dtype, [&](auto* tag) {
            using T = std::remove_pointer_t<decltype(tag)>;
            return compress_t<T>(psi, opts, out, alloc, stream);
        });
    })
}

thc_status mps_inner(const thc_mps* phi, const thc_mps* psi, double* out_re, double* out_im, void* stream) {
    THC_GUARD({
        check_mps(phi, "phi");
        check_mps(psi, "psi");
        if (phi->L != psi->L) throw Error(THC_EINVAL, "L mismatch");
        if (phi->dtype != psi->dtype) throw Error(THC_EINVAL, "dtype mismatch");
        if (!out_re) throw Error(THC_EINVAL, "null output");
        return dispatch(phi->dtype, [&](auto* tag) {
            using T = std::remove_pointer_t<decltype(tag)>;
            return inner_t<T>(phi, psi, out_re, out_im, stream);
        });
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
            if (xs[i]->dtype != xs[0]->dtype) throw Error(THC_EINVAL, "dtype mismatch");
        }
        check_complex_dmax(xs[0]->dtype, opts);
        if (coeff_im && !is_complex(xs[0]->dtype))
            for (int i = 0; i < n; ++i)
                if (coeff_im[i] != 0.0) throw Error(THC_EINVAL, "complex coefficients need complex MPS");
        return dispatch(xs[0]->dtype, [&](auto* tag) {
            using T = std::remove_pointer_t<decltype(tag)>;
            return add_t<T>(n, coeff_re, coeff_im, xs, opts, out, alloc, stream);
        });
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
        check_complex_dmax(psi0->dtype, opts);
        if (K < 1 || K > thc::SMALL_MAX) throw Error(THC_EINVAL, "K must be in [1, 64]");
        if (!energy) throw Error(THC_EINVAL, "null energy");
        return dispatch(psi0->dtype, [&](auto* tag) {
            using T = std::remove_pointer_t<decltype(tag)>;
            return lanczos_t<T>(H, psi0, K, opts, energy, ritz, ground, alloc, stream);
        });
    })
}

thc_status krylov_lanczos_restarted(const thc_hamiltonian* H, const thc_mps* psi0, int K, int cycles, int n_lower,
                                    const thc_mps* const* lower, const thc_opts* opts, double* energies,
                                    thc_mps* state, const thc_allocator* alloc, void* stream) {
    THC_GUARD({
        check_mps(psi0, "psi0");
        check_opts(opts);
        check_ham(H, psi0->L);
        check_path_dtype(psi0, opts);
        check_complex_dmax(psi0->dtype, opts);
        if (K < 1 || K > thc::SMALL_MAX) throw Error(THC_EINVAL, "K must be in [1, 64]");
        if (cycles < 1) throw Error(THC_EINVAL, "cycles must be >= 1");
        if (n_lower < 0 || (n_lower > 0 && !lower)) throw Error(THC_EINVAL, "bad lower states");
        if (!energies) throw Error(THC_EINVAL, "null energies");
        for (int m = 0; m < n_lower; ++m) {
            check_mps(lower[m], "lower");
            if (lower[m]->L != psi0->L || lower[m]->dtype != psi0->dtype)
                throw Error(THC_EINVAL, "lower states must match psi0's L and dtype");
        }
        return dispatch(psi0->dtype, [&](auto* tag) {
            using T = std::remove_pointer_t<decltype(tag)>;
            return restarted_t<T>(H, psi0, K, cycles, n_lower, lower, opts, energies, state, alloc, stream);
        });
    })
}

thc_status thc_expect_grad(const thc_hamiltonian* H, const thc_mps* phi, const thc_mps* psi, const thc_opts* opts,
                           double* value, double* grad_t, double* grad_chi, double* grad_zeta, thc_mps* grad_psi,
                           const thc_allocator* alloc, void* stream) {
    THC_GUARD({
        check_mps(phi, "phi");
        check_mps(psi, "psi");
        check_opts(opts);
        check_ham(H, psi->L);
        check_path_dtype(psi, opts);
        if (phi->L != psi->L || phi->dtype != psi->dtype) throw Error(THC_EINVAL, "phi and psi differ in L or dtype");
        if (is_complex(psi->dtype)) throw Error(THC_EUNSUPPORTED, "the adjoint is built for real MPS");
        if (!value) throw Error(THC_EINVAL, "null value");
        if (psi->dtype == THC_F64)
            return expect_grad_t<double>(H, phi, psi, opts, value, grad_t, grad_chi, grad_zeta, grad_psi, alloc,
                                         stream);
        return expect_grad_t<float>(H, phi, psi, opts, value, grad_t, grad_chi, grad_zeta, grad_psi, alloc, stream);
    })
}

thc_status krylov_expm_apply(const thc_hamiltonian* H, const thc_mps* psi, double dt, int K,
                             const thc_opts* opts, thc_mps* out, double* lost_norm,
                             const thc_allocator* alloc, void* stream) {
    THC_GUARD({
        check_mps(psi, "psi");
        check_opts(opts);
        check_ham(H, psi->L);
        check_path_dtype(psi, opts);
        check_complex_dmax(complex_dtype(opts->path), opts);
        if (K < 1 || K > thc::SMALL_MAX) throw Error(THC_EINVAL, "K must be in [1, 64]");
        if (!out) throw Error(THC_EINVAL, "null output");
        if (!std::isfinite(dt)) throw Error(THC_EINVAL, "dt must be finite");
        if (opts->path == THC_PATH_FP64) return expm_t<c64>(H, psi, dt, K, opts, out, lost_norm, alloc, stream);
        return expm_t<c32>(H, psi, dt, K, opts, out, lost_norm, alloc, stream);
    })
}

thc_status thc_kinetic_factors(int L, const double* t, double* lambda, double* u, void* stream) {
    THC_GUARD({
        if (L < 1 || L > thc::SMALL_MAX || !t || !lambda || !u) throw Error(THC_EINVAL, "bad arguments");
        const cudaStream_t st = (cudaStream_t)stream;
        thc::Alloc al;
        al.st = st;
        Scratch sc(al);
        int* flag = sc.get<int>(1);
        THC_CUDA(cudaFuncSetAttribute(thc::k_kinetic_factors, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)thc::KINETIC_SMEM));
        THC_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
        {
            THC_LAUNCH("kinetic_eigh", st);
            thc::k_kinetic_factors<<<1, 256, thc::KINETIC_SMEM, st>>>(L, t, lambda, u, flag);
        }
        THC_CUDA(cudaGetLastError());
        int f = 0;
        THC_CUDA(cudaMemcpyAsync(&f, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        THC_CUDA(cudaStreamSynchronize(st));
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
