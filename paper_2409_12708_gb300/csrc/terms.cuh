// terms.cuh -- the Coulomb term list of Eq. G as index arithmetic (no
// dependencies: host code and tests include it as plain C++).
#pragma once

#ifdef __CUDACC__
#define THC_HD __host__ __device__
#else
#define THC_HD
#endif

namespace thc {

// Coulomb term list (Eq. G).  Unmerged: t = ((s'*N + nu)*2 + s)*N + mu, 4N^2
// terms.  Spin-merged (symmetric zeta): the opposite-spin pair (mu down, nu up)
// is folded into (mu up, nu down), which commute and carry the same zeta; the
// list is block (nu, up) with mu up only (t < N^2), then block (nu, down)
// with s = up (factor 2) and s = down, 3N^2 terms.  block = s'*N + nu is the
// index of the reused state psi_{nu s'}.
struct TermIdx {
    int mu, s, nu, sp;
    double factor;
};
THC_HD inline long coulomb_terms(int N, int merge) { return (merge ? 3L : 4L) * N * N; }
THC_HD inline TermIdx decode_coulomb(long t, int N, int merge) {
    TermIdx d;
    d.factor = 1.0;
    if (!merge) {
        d.mu = (int)(t % N);
        long rest = t / N;
        d.s = (int)(rest % 2);
        rest /= 2;
        d.nu = (int)(rest % N);
        d.sp = (int)(rest / N);
    } else if (t < (long)N * N) {
        d.mu = (int)(t % N);
        d.s = 0;
        d.nu = (int)(t / N);
        d.sp = 0;
    } else {
        const long k = t - (long)N * N;
        d.mu = (int)(k % N);
        d.s = (int)((k / N) % 2);
        d.nu = (int)(k / (2L * N));
        d.sp = 1;
        if (d.s == 0) d.factor = 2.0;
    }
    return d;
}
THC_HD inline long coulomb_block(long t, int N, int merge) {
    const TermIdx d = decode_coulomb(t, N, merge);
    return (long)d.sp * N + d.nu;
}

}  // namespace thc
