// engine_impl.cuh -- Engine<T>: the hot path of the THC-MPO method on one GPU.
#pragma once

#include "engine.cuh"

namespace thc {

static __global__ void k_pair_src(int* a, int* b, int B, int start) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B) {
        a[i] = start + 2 * i;
        b[i] = start + 2 * i + 1;
    }
}

// Per-wave scratch for all plans of one call (sized by the largest plan).
template <class T>
struct Work {
    int B = 0;
    long sWide = 0, sL = 0, sC = 0, sZ = 0, sV = 0, sTw = 0, sSv = 0;
    long sTwSite = 0;  // T matrices of one site's QR; sTw = sites x sTwSite per term
    T *wide = nullptr, *Lb[2] = {nullptr, nullptr}, *C = nullptr, *W = nullptr, *Z = nullptr;
    T *V = nullptr, *M[2] = {nullptr, nullptr}, *Tw = nullptr;
    double* sv = nullptr;
    int* keep = nullptr;
    T* nu = nullptr;  // column norms of U (stride sSv)
    T* F = nullptr;   // V V^T (stride sF)
    long sF = 0;
    int* perm = nullptr;  // column order of C for the pivoted preconditioning QR
    long sPerm = 0;
    // per-term layer data
    T *coef1 = nullptr, *coef2 = nullptr, *pcoef = nullptr;
    int *op1 = nullptr, *op2 = nullptr, *src = nullptr, *srcA = nullptr, *srcB = nullptr;
};

template <class T>
struct Engine {
    cudaStream_t st;
    Alloc al;
    int* dflag = nullptr;  // device status word
    double* ddbg = nullptr;  // device diagnostics of a non-converged Jacobi ([4])
    int sms = 152;
    int smem_optin = 227 * 1024;  // largest dynamic shared memory a block may opt in to

    Engine(cudaStream_t s, const thc_allocator* a) : st(s) {
        al.a = a;
        al.st = s;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        static std::once_flag attrs_once;  // engines may be built on several host threads
        std::call_once(attrs_once, set_attrs);
    }

    // Opt in to large dynamic shared memory: the per-block limit minus the
    // kernel's static shared memory.
    template <class K>
    static void opt_in(K kern, int want) {
        cudaFuncAttributes fa;
        THC_CUDA(cudaFuncGetAttributes(&fa, kern));
        int dev = 0, optin = 0;
        THC_CUDA(cudaGetDevice(&dev));
        THC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        const int v = std::min<int>(want, optin - (int)fa.sharedSizeBytes);
        THC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
    }
    static void set_attrs() {
        const int big = 1 << 30;
        opt_in(k_qr<T>, big);
        opt_in(k_jacobi_select<T, 4>, big);
        opt_in(k_jacobi_select<T, 8>, big);
        opt_in(k_jacobi_select<T, 16>, big);
        if constexpr (!is_complex_v<T>) opt_in(k_jacobi_select<T, 32>, big);
        opt_in(k_kinetic_factors, (int)KINETIC_SMEM);
        opt_in(k_krylov_small, (int)KRYLOV_SMEM);
        opt_in(k_krylov_small_c, (int)KRYLOV_SMEM_C);
        if constexpr (std::is_same<T, float>::value) opt_in(k_apply_qt, big);
    }

    void check() { THC_CUDA(cudaGetLastError()); }

    bool tc = false;  // TF32 path: float32 contractions on the tensor cores (3xTF32)

    // Batched GEMM of the compression.  On the TF32 path (float32 storage,
    // output at least 64 x 64) a small autotuner picks the kernel: the first
    // time a contraction of one kind (loader and store types) and shape, with a
    // batch in one power-of-two bucket, runs in the process, the tensor-core
    // and the SIMT kernel both run it and are timed with CUDA events; the
    // faster is remembered for that key and run once more, so the output always
    // comes from the kernel chosen.  Otherwise the SIMT kernels.
    template <class LA, class LB, class SC>
    void gemm(int batch, int M, int N, int K, const LA& la, const LB& lb, const SC& sc) {
        if constexpr (std::is_same<T, float>::value) {
            if (tc && batch > 0 && M >= 64 && N >= 64 && K >= 1) {
                static std::once_flag attr_once;  // one opt-in per instantiation
                std::call_once(attr_once, [] {
                    THC_CUDA(cudaFuncSetAttribute(k_gemm_tc<LA, LB, SC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  tc::SMEM));
                });
                auto run_tc = [&] {
                    dim3 grid(ceil_div(N, tc::BN), ceil_div(M, tc::BM), batch);
                    k_gemm_tc<LA, LB, SC><<<grid, tc::THREADS, tc::SMEM, st>>>(M, N, K, la, lb, sc, dflag);
                    THC_CUDA(cudaGetLastError());
                    Profiler& p = profiler();
                    if (p.on) {  // every contraction run on the tensor cores, tuning runs included
                        std::lock_guard<std::mutex> g(p.mu);
                        p.acc["tc_gemm_launches"].first += 1;
                    }
                };
                auto run_simt = [&] { THC_CUDA(launch_gemm<T>(batch, M, N, K, la, lb, sc, st)); };
                int bucket = 0;
                while ((1 << bucket) < batch) ++bucket;
                const GemmKey key{typeid(k_gemm_tc<LA, LB, SC>).hash_code(), M, N, K, bucket};
                int pick = tuned(key);
                if (pick < 0) {
                    cudaEvent_t e[3];
                    for (auto& x : e) THC_CUDA(cudaEventCreate(&x));
                    THC_CUDA(cudaEventRecord(e[0], st));
                    run_tc();
                    THC_CUDA(cudaEventRecord(e[1], st));
                    run_simt();
                    THC_CUDA(cudaEventRecord(e[2], st));
                    THC_CUDA(cudaEventSynchronize(e[2]));
                    float t_tc = 0.f, t_simt = 0.f;
                    THC_CUDA(cudaEventElapsedTime(&t_tc, e[0], e[1]));
                    THC_CUDA(cudaEventElapsedTime(&t_simt, e[1], e[2]));
                    for (auto& x : e) cudaEventDestroy(x);
                    pick = t_tc <= t_simt ? 1 : 0;
                    remember(key, pick);
                }
                if (pick == 1) run_tc();
                else run_simt();
                return;
            }
        }
        THC_CUDA(launch_gemm<T>(batch, M, N, K, la, lb, sc, st));
    }

    // the autotuner's table: kernel kind and shape -> 1 (tensor cores) or 0 (SIMT)
    struct GemmKey {
        size_t kind;
        int M, N, K, bucket;
        bool operator<(const GemmKey& o) const {
            return std::tie(kind, M, N, K, bucket) < std::tie(o.kind, o.M, o.N, o.K, o.bucket);
        }
    };
    static std::mutex& tune_mu() {
        static std::mutex m;
        return m;
    }
    static std::map<GemmKey, int>& tune_table() {
        static std::map<GemmKey, int> t;
        return t;
    }
    static int tuned(const GemmKey& k) {
        std::lock_guard<std::mutex> g(tune_mu());
        auto it = tune_table().find(k);
        return it == tune_table().end() ? -1 : it->second;
    }
    static void remember(const GemmKey& k, int pick) {
        std::lock_guard<std::mutex> g(tune_mu());
        tune_table()[k] = pick;
    }

    // ---------------------------------------------------------------- work
    void alloc_work(Scratch& sc, Work<T>& w, int B, const std::vector<const Plan*>& plans) {
        Plan mx;
        for (auto* p : plans) {
            mx.wsize = std::max(mx.wsize, p->wsize);
            mx.maxL = std::max(mx.maxL, p->maxL);
            mx.maxC = std::max(mx.maxC, p->maxC);
            mx.maxZ = std::max(mx.maxZ, p->maxZ);
            mx.maxV = std::max(mx.maxV, p->maxV);
            mx.maxTw = std::max(mx.maxTw, p->maxTw);
            mx.maxKout = std::max(mx.maxKout, p->maxKout);
        }
        w.B = B;
        // per-term strides rounded up to 128 bytes: every term's matrices stay aligned
        auto up = [](long x) { return (std::max(1L, x) + 31) / 32 * 32; };
        w.sWide = up(mx.wsize);
        w.sL = up(mx.maxL);
        w.sC = up(mx.maxC);
        w.sZ = up(mx.maxZ);
        w.sV = up(mx.maxV);
        // every site keeps its QR's T matrices until the SVD sweep applies its Q
        const long sites = plans.empty() ? 1 : std::max(1, plans[0]->L);
        w.sTwSite = up(mx.maxTw);
        w.sTw = sites * w.sTwSite;
        w.sSv = up(mx.maxKout);
        w.wide = sc.get<T>((size_t)B * w.sWide);
        w.Lb[0] = sc.get<T>((size_t)B * w.sL);
        w.Lb[1] = sc.get<T>((size_t)B * w.sL);
        w.C = sc.get<T>((size_t)B * w.sC);
        w.W = sc.get<T>((size_t)B * w.sC);
        w.Z = sc.get<T>((size_t)B * w.sZ);
        w.V = sc.get<T>((size_t)B * w.sV);
        w.M[0] = sc.get<T>((size_t)B * w.sV);
        w.M[1] = sc.get<T>((size_t)B * w.sV);
        w.Tw = sc.get<T>((size_t)B * w.sTw);
        w.sv = sc.get<double>((size_t)B * w.sSv);
        w.nu = sc.get<T>((size_t)B * w.sSv);
        w.sF = up(mx.maxKout * mx.maxKout);
        w.F = sc.get<T>((size_t)B * w.sF);
        w.keep = sc.get<int>((size_t)B);
        long maxN = 1;
        for (auto* p : plans) maxN = std::max<long>(maxN, p->maxN);
        w.sPerm = maxN;
        w.perm = sc.get<int>((size_t)B * maxN);
        const int L = plans.empty() ? 1 : plans[0]->L;
        w.coef1 = sc.get<T>((size_t)B * L);
        w.coef2 = sc.get<T>((size_t)B * L);
        w.pcoef = sc.get<T>((size_t)2 * B);
        w.op1 = sc.get<int>((size_t)B);
        w.op2 = sc.get<int>((size_t)B);
        w.src = sc.get<int>((size_t)B);
        w.srcA = sc.get<int>((size_t)B);
        w.srcB = sc.get<int>((size_t)B);
    }

    static size_t work_bytes_per_term(const std::vector<const Plan*>& plans) {
        long wsize = 0, maxL = 0, maxC = 0, maxZ = 0, maxV = 0, maxTw = 0, kout = 0;
        int L = 1;
        for (auto* p : plans) {
            wsize = std::max(wsize, p->wsize);
            maxL = std::max(maxL, p->maxL);
            maxC = std::max(maxC, p->maxC);
            maxZ = std::max(maxZ, p->maxZ);
            maxV = std::max(maxV, p->maxV);
            maxTw = std::max(maxTw, p->maxTw);
            kout = std::max(kout, p->maxKout);
            L = p->L;
        }
        return sizeof(T) * (size_t)(wsize + 2 * maxL + 2 * maxC + maxZ + 3 * maxV + (long)L * maxTw + 2 * L + 2) +
               sizeof(double) * kout + 8 * sizeof(int);
    }

    // ------------------------------------------------------------ compress
    // Expand (bond-2 MPO layer or direct sum) and compress a batch of B terms.
    // ex: loader with the term-level fields set (mode, inputs, coefficients);
    // the per-site fields are filled here.  Output: out + b*out_stride, profile P.out.
    void compress(const Plan& P, int B, ExpandA<T> ex, T* out, long out_stride, Work<T>& w) {
        const int L = P.L;
        if (L < 2) throw Error(THC_EINVAL, "L >= 2 required");
        Profile pA(P.inA), pO(P.out);
        Profile pB = P.mode == MODE_DIRSUM ? Profile(P.inB) : Profile();
        ex.L = L;
        // sites whose Q is applied to M_{s-1} in the SVD sweep instead of being
        // formed (real float32, 32-column panels, m <= 1024)
        std::vector<char> qt(L + 1, 0);
        // ---- QR sweep, right to left: X_s = expand(site s) * L_{s+1}; X_s = L_s Q_s
        for (int s = L - 1; s >= 0; --s) {
            ex.s = s;
            ex.offA = pA.off[s];
            ex.lA = P.inA[s];
            ex.rA = P.inA[s + 1];
            if (P.mode == MODE_DIRSUM) {
                ex.offB = pB.off[s];
                ex.lB = P.inB[s];
                ex.rB = P.inB[s + 1];
            }
            ex.rows0 = P.inA[s];
            ex.cols0 = (s == L - 1) ? 1 : P.inA[s + 1];
            const int Mg = P.e[s] * 4, Ng = P.k[s + 1], Kg = P.e[s + 1];
            RowMajorB<T> bop{s == L - 1 ? nullptr : w.Lb[(s + 1) & 1], w.sL, P.k[s + 1]};
            StoreRM<T> sto{w.wide + P.woff[s], w.sWide, Ng};
            {
                THC_LAUNCH("gemm_expand_absorb", st);
                gemm(B, Mg, Ng, Kg, ex, bop, sto);
            }
            if (s >= 1) {
                QRJob<T> job;
                job.A = w.wide + P.woff[s];
                job.strideA = w.sWide;
                job.m = 4 * P.k[s + 1];
                job.n = P.e[s];
                job.ld = job.m;
                job.Tw = w.Tw + (long)s * w.sTwSite;
                job.strideT = w.sTw;
                job.out = w.Lb[s & 1];
                job.strideOut = w.sL;
                qr_params<T>(job.m, job.n, job.nb);
                if constexpr (std::is_same<T, float>::value)
                    qt[s] = job.nb == QT_NB && job.m <= 1024 && (int)qt_smem_bytes(job.m) <= smem_optin - 2048;
                job.mode = qt[s] ? QR_L_ONLY : QR_L_AND_Q;
                job.colmap = nullptr;
                job.pivot = 0;
                {
                    THC_LAUNCH("qr_lq_sweep", st);
                    k_qr<T><<<B, QR_THREADS, qr_smem_bytes<T>(job.m, job.nb, job.n), st>>>(job);
                }
                check();
            }
        }
        // ---- SVD sweep, left to right
        for (int s = 0; s < L - 1; ++s) {
            const int m = 4 * P.out[s], n = P.k[s + 1], kout = P.out[s + 1];
            // C_s = M_{s-1} Q_s  (M_{-1} = [1], Q_0 = X_0)
            StoreC<T> sto{w.C, w.sC, m >= n ? w.W : nullptr, w.sC, m, n, 4 * n};
            RowMajorB<T> qop{w.wide + P.woff[s], w.sWide, 4 * n};
            if (s == 0) {
                THC_LAUNCH("gemm_center", st);
                gemm(B, P.out[0], 4 * n, 1, IdentA<T>{}, qop, sto);
            } else if (qt[s]) {
                THC_LAUNCH("qt_apply", st);
                apply_qt(B, P, s, w, w.C, w.sC, 4 * n, m >= n ? w.W : nullptr, n);
            } else {
                RowMajorA<T> mop{w.M[(s - 1) & 1], w.sV, P.k[s]};
                THC_LAUNCH("gemm_center", st);
                gemm(B, P.out[s], 4 * n, P.k[s], mop, qop, sto);
            }
            int p = std::min(m, n);
            const int* colmap = nullptr;
            if (m >= n) {
                // block-pivoted QR (square factors too: an unpivoted square C with a
                // numerically null part can take the Jacobi past its sweep budget):
                // the kernel writes the column order it chose to w.perm
                colmap = w.perm;
                QRJob<T> job;
                job.colmap = w.perm;
                job.pivot = 1;
                job.A = w.W;
                job.strideA = w.sC;
                job.m = m;
                job.n = n;
                job.ld = m;
                job.Tw = w.Tw;
                job.strideT = w.sTw;
                job.out = w.Z;
                job.strideOut = w.sZ;
                qr_params<T>(m, n, job.nb);
                job.mode = QR_R_ROWS;
                {
                    THC_LAUNCH("qr_svd_precond", st);
                    k_qr<T><<<B, QR_THREADS, qr_smem_bytes<T>(m, job.nb, n), st>>>(job);
                }
                check();
            } else {
                dim3 g(ceil_div(m * n, 256 * 4) + 1, B);
                THC_LAUNCH("copy", st);
                k_copy_batched<T><<<g, 256, 0, st>>>(w.Z, w.sZ, w.C, w.sC, (long)m * n);
                check();
            }
            jacobi_select(B, p, n, kout, w, colmap);
            // U = C V^T -> output site s, then normalise and form M_s
            RowMajorA<T> cop{w.C, w.sC, n};
            TransB<T> vop{w.V, w.sV, n};
            StoreRM<T> uo{out + pO.off[s], out_stride, kout};
            {
                THC_LAUNCH("gemm_u", st);
                gemm(B, m, kout, n, cop, vop, uo);
            }
            // normalise U's columns, then M = diag(nu) (I - F') V with F = V V^T
            {
                THC_LAUNCH("svd_finalize", st);
                dim3 g(ceil_div(kout, 128), B);
                k_unit_columns<T><<<g, 128, 0, st>>>(out + pO.off[s], out_stride, m, kout, w.nu, w.sSv);
            }
            check();
            {
                THC_LAUNCH("svd_finalize", st);
                gemm(B, kout, kout, n, RowMajorA<T>{w.V, w.sV, n}, TransB<T>{w.V, w.sV, n},
                                        StoreRM<T>{w.F, w.sF, kout});
            }
            {
                THC_LAUNCH("svd_finalize", st);
                gemm(B, kout, n, kout, CorrA<T>{w.F, w.sF, w.nu, w.sSv, kout},
                                        RowMajorB<T>{w.V, w.sV, n}, StoreRM<T>{w.M[s & 1], w.sV, n});
            }
        }
        // ---- last site: M_{L-2} Q_{L-1}
        {
            const int s = L - 1;
            if (qt[s]) {
                THC_LAUNCH("qt_apply", st);
                apply_qt(B, P, s, w, out + pO.off[s], out_stride, 4 * P.k[s + 1], nullptr, 1);
            } else {
                RowMajorA<T> mop{w.M[(s - 1) & 1], w.sV, P.k[s]};
                RowMajorB<T> qop{w.wide + P.woff[s], w.sWide, 4 * P.k[s + 1]};
                StoreRM<T> so{out + pO.off[s], out_stride, 4 * P.k[s + 1]};
                THC_LAUNCH("gemm_center", st);
                gemm(B, P.out[s], 4 * P.k[s + 1], P.k[s], mop, qop, so);
            }
        }
    }

    // C = M_{s-1} Q_s from the reflectors the QR sweep left at site s (real
    // float32 only; qt_apply.cuh)
    void apply_qt(int B, const Plan& P, int s, Work<T>& w, T* C, long strideC, int ldC, T* W, int nW) {
        if constexpr (std::is_same<T, float>::value) {
            QtJob<float> j;
            j.M = w.M[(s - 1) & 1];
            j.strideM = w.sV;
            j.ldM = P.k[s];
            j.A = w.wide + P.woff[s];
            j.strideA = w.sWide;
            j.ld = 4 * P.k[s + 1];
            j.Tw = w.Tw + (long)s * w.sTwSite;
            j.strideT = w.sTw;
            j.out = P.out[s];
            j.m = 4 * P.k[s + 1];
            j.kk = P.k[s];
            j.C = C;
            j.strideC = strideC;
            j.ldC = ldC;
            j.W = W;
            j.strideW = w.sC;
            j.nW = nW;
            dim3 g(ceil_div(j.out, QT_RB), B);
            k_apply_qt<<<g, QT_THREADS, qt_smem_bytes(j.m), st>>>(j);
            check();
        } else {
            (void)B; (void)P; (void)s; (void)w; (void)C; (void)strideC; (void)ldC; (void)W; (void)nW;
            throw Error(THC_EINVAL, "reflector application is float32 only");
        }
    }

    // rotation threshold on the row cosine: a multiple of the rounding error of
    // the warp dot product (NPL sequential terms per lane + 5 butterfly levels)
    double rot_tol(int n) const { return 8.0 * (ceil_div(std::max(n, 1), 32) + 6) * Real<real_t<T>>::eps; }
    double tol_ = 0.0;

    void jacobi_select(int B, int p, int n, int kout, Work<T>& w, const int* colmap) {
        JacobiJob<T> j;
        j.Z = w.Z;
        j.strideZ = w.sZ;
        j.p = p;
        j.n = n;
        j.V = w.V;
        j.strideV = w.sV;
        j.sv = w.sv;
        j.strideSv = w.sSv;
        j.keep = w.keep;
        j.kout = kout;
        j.tol = tol_;
        j.rot_tol = rot_tol(n);
        j.max_sweeps = 30;
        j.status = dflag;
        j.dbg = ddbg;
        j.colmap = colmap;
        // rows of Z that fit in shared memory next to sigma^2 and the order
        const size_t budget = (size_t)std::min(224 * 1024, smem_optin - 2048);
        const size_t base = ((size_t)p * (sizeof(double) + sizeof(int)) + 15) & ~(size_t)15;
        const size_t row = (size_t)n * sizeof(T);
        j.ps = (int)std::min<size_t>((size_t)p, (budget - base) / row);
        const size_t smem = base + (size_t)j.ps * row;
        THC_LAUNCH("jacobi_svd", st);
        if (n <= 128) k_jacobi_select<T, 4><<<B, JacobiCfg<T, 4>::threads, smem, st>>>(j);
        else if (n <= 256) k_jacobi_select<T, 8><<<B, JacobiCfg<T, 8>::threads, smem, st>>>(j);
        else if (n <= 512) k_jacobi_select<T, 16><<<B, JacobiCfg<T, 16>::threads, smem, st>>>(j);
        else if constexpr (!is_complex_v<T>) {
            if (n <= 1024) k_jacobi_select<T, 32><<<B, JacobiCfg<T, 32>::threads, smem, st>>>(j);
            else throw Error(THC_EUNSUPPORTED, "bond dimension above 512 is not supported");
        } else {
            throw Error(THC_EUNSUPPORTED, "complex MPS: bond dimension above 256 is not supported");
        }
        check();
    }

    // ---------------------------------------------------------- reduction
    // Pairwise add-and-compress of n MPS (profile prof) stored at buf; result
    // returned in a buffer from sc (or buf itself when n == 1).
    T* reduce(Scratch& sc, T* buf, long n, const std::vector<int>& prof, int D, int Bw) {
        Profile pf(prof);
        Plan PD = make_plan<T>(MODE_DIRSUM, prof, prof, D);
        for (int b = 0; b <= pf.L; ++b)
            if (PD.out[b] != prof[b]) throw Error(THC_EINVAL, "reduction profile is not a fixed point");
        if (n == 1) return buf;
        const long half = (n + 1) / 2;
        T* nxt0 = sc.get<T>((size_t)half * pf.size);
        T* nxt1 = half > 1 ? sc.get<T>((size_t)((half + 1) / 2) * pf.size) : nullptr;
        Scratch ws(al);
        Work<T> w;
        const int B = (int)std::min<long>(Bw, n / 2);
        alloc_work(ws, w, B, {&PD});
        {
            THC_LAUNCH("setup", st);
            k_pair_coefs<T><<<ceil_div(B, 128), 128, 0, st>>>(w.pcoef, B, nullptr, nullptr);
        }
        check();
        T* cur = buf;
        int flip = 0;
        while (n > 1) {
            const long np = n / 2;
            T* nxt = flip ? nxt1 : nxt0;
            for (long j0 = 0; j0 < np; j0 += B) {
                const int Bc = (int)std::min<long>(B, np - j0);
                {
                    THC_LAUNCH("setup", st);
                    k_pair_src<<<ceil_div(Bc, 128), 128, 0, st>>>(w.srcA, w.srcB, Bc, (int)(2 * j0));
                }
                check();
                ExpandA<T> ex{};
                ex.mode = MODE_DIRSUM;
                ex.inA = cur;
                ex.strideA = pf.size;
                ex.srcA = w.srcA;
                ex.inB = cur;
                ex.strideB = pf.size;
                ex.srcB = w.srcB;
                ex.coef = w.pcoef;
                compress(PD, Bc, ex, nxt + j0 * pf.size, pf.size, w);
            }
            if (n & 1)
                THC_CUDA(cudaMemcpyAsync(nxt + np * pf.size, cur + (n - 1) * pf.size, pf.size * sizeof(T),
                                         cudaMemcpyDeviceToDevice, st));
            cur = nxt;
            n = (n + 1) / 2;
            flip ^= 1;
        }
        return cur;
    }
};

}  // namespace thc
