// tc_gemm.cuh -- batched float32 GEMM on the 5th-generation tensor cores
// (tcgen05.mma kind::tf32, accumulators in tensor memory), with the error-
// compensated split of Ootomo & Yokota (2022): each float32 operand is the sum
// of two TF32 numbers, a = a_hi + a_lo, and C = A_hi B_hi + A_hi B_lo + A_lo B_hi
// reaches float32 accuracy (the dropped A_lo B_lo term is ~2^-22 of the
// product).  The tensor core adds into its float32 accumulator with rounding
// toward zero; accumulated over a whole K that bias shrinks every product by
// ~K ulps, and a compression chains enough products for it to show (measured:
// -4e-4 in |H psi|^2 over 16 terms).  So, as in that paper, accumulation across
// K happens outside the tensor core: every 32-wide K slice is accumulated in a
// fresh pair of tensor-memory accumulators (A_hi B_hi, and the two correction
// products), which the threads read back and add into float32 registers with
// round-to-nearest.
//
// C[b](m, n) = sum_k A[b](m, k) B[b](k, n), operands produced element by
// element by loader functors (the bond-2 MPO expansion and the direct sum stay
// fused into the operand load), C written by a store functor.  One CTA of 256
// threads per 128 x 128 tile of C (blockIdx.z = batch):
//   * the threads load the 128 x 32 slices of A and B^T into registers (each
//     thread 4 rows' 4-element k-chunks of each), split them, and store them in
//     the no-swizzle K-major canonical layout (8-row x 16-byte core matrices;
//     k-chunks 128 bytes apart, 8-row groups 1 KB apart) with 16-byte stores
//     that fill 512 contiguous bytes per warp; two stages; the loads of
//     slice k+1 are issued right after the MMAs of slice k, so their latency
//     overlaps the tensor core's work and the read-back below;
//   * one thread issues the 12 MMAs of a slice (K = 8 each) into the slice's
//     accumulator pair and commits them to the stage's mbarrier;
//   * while the tensor core works on slice k, the threads read back slice
//     k-1's accumulators (tcgen05.ld; warp w: lanes 32 (w % 4) .., columns
//     64 (w / 4) ..) and add them to their registers; the pairs alternate, so
//     tensor memory holds 4 x 128 columns.
// Waits on an mbarrier are bounded (one second by %globaltimer); a wait that
// gives up sets DEV_TC_TIMEOUT in the status word, skips the epilogue, and the
// CTA still releases its tensor memory before it returns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace thc {

namespace tc {

constexpr int BM = 128, BN = 128, BK = 32, THREADS = 256;
constexpr uint32_t LBO = 128;              // bytes between k-chunks (4 float32) of one core matrix row group
constexpr uint32_t SBO = (BK / 4) * 128;   // bytes between 8-row groups
constexpr int PART = BM * BK * 4;          // one operand part (hi or lo) of one stage: 16 KB
constexpr int STAGE = 4 * PART;            // A_hi, A_lo, B_hi, B_lo
constexpr int SMEM = 2 * STAGE + 1024;     // two stages + alignment slack
// instruction descriptor: float32 accumulator, TF32 A and B, both K-major, N = 128, M = 128
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
constexpr uint32_t TMEM_COLS = 512;  // 2 slices in flight x (hi product, corrections) x 128 columns

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// byte offset of element (row r, k) of a 128 x 32 slice in the canonical layout
__device__ __forceinline__ uint32_t kmaj_off(int r, int k) {
    return (uint32_t)((r >> 3) * SBO + (k >> 2) * LBO + (r & 7) * 16 + (k & 3) * 4);
}

// shared-memory matrix descriptor: start address, LBO, SBO, version 1, no swizzle
__device__ __forceinline__ uint64_t desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)(SBO >> 4) << 32) |
           ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(tmem),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}

// wait for the phase of the given parity to complete; false after one second
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (long it = 0; it < (1L << 26); ++it) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(mbar), "r"(parity));
        if (done) return true;
        if ((it & 255) == 255) {
            uint64_t t1;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
            if (t1 - t0 > 1000000000ull) return false;
        }
    }
    return false;
}

template <int I>
__device__ __forceinline__ void ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
          "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}

}  // namespace tc

template <class LA, class LB, class SC>
__global__ void __launch_bounds__(tc::THREADS, 1)
k_gemm_tc(int M, int N, int K, LA la, LB lb, SC sc, int* status) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) &
                                                           ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.z, m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_sh;
    const int nkt = (K + BK - 1) / BK;
    // this thread's share of the accumulator: row lane_base + lane, 64 columns
    const int lane_base = 32 * (warp & 3), col_base = 64 * (warp >> 2);
    float acc[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) acc[j] = 0.f;
    // loads: lane -> (row (lane & 7) of an 8-row group, k-chunk (lane >> 3) of a quad);
    // warp w, step j -> 8-row group 2 j + (w >> 2) ... so the 8 warps x 4 steps cover
    // 16 row groups x 2 chunk quads
    const int lr = lane & 7, lc = lane >> 3;
    uint32_t parity[2] = {0u, 0u};
    bool ok = true;
    // this thread's elements of slice kt: va/vb[j][e] = A(m0 + r, k) and B(k, n0 + r)
    float va[4][4], vb[4][4];
    auto load_slice = [&](int kt) {
        const int k0 = kt * BK;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int unit = warp * 4 + j;            // 0..31
            const int g = unit >> 1, q = unit & 1;    // row group, chunk quad
            const int r = g * 8 + lr, c = q * 4 + lc; // row in tile, k-chunk in slice
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = k0 + 4 * c + e;
                va[j][e] = (m0 + r < M && k < K) ? (float)la(b, m0 + r, k) : 0.f;
                vb[j][e] = (n0 + r < N && k < K) ? (float)lb(b, k, n0 + r) : 0.f;
            }
        }
    };
    if (nkt > 0) load_slice(0);
    for (int kt = 0; kt < nkt && ok; ++kt) {
        const int st = kt & 1;
        unsigned char* a_hi = smem + st * STAGE;
        unsigned char* a_lo = a_hi + PART;
        unsigned char* b_hi = a_hi + 2 * PART;
        unsigned char* b_lo = a_hi + 3 * PART;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int unit = warp * 4 + j;
            const int g = unit >> 1, q = unit & 1;
            const int r = g * 8 + lr, c = q * 4 + lc;
            const uint32_t off = kmaj_off(r, 4 * c);
            uint4 ah, al, bh, bl;
            uint32_t* pah = reinterpret_cast<uint32_t*>(&ah);
            uint32_t* pal = reinterpret_cast<uint32_t*>(&al);
            uint32_t* pbh = reinterpret_cast<uint32_t*>(&bh);
            uint32_t* pbl = reinterpret_cast<uint32_t*>(&bl);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                pah[e] = tf32_rna(va[j][e]);
                pal[e] = tf32_rna(va[j][e] - __uint_as_float(pah[e]));
                pbh[e] = tf32_rna(vb[j][e]);
                pbl[e] = tf32_rna(vb[j][e] - __uint_as_float(pbh[e]));
            }
            *reinterpret_cast<uint4*>(a_hi + off) = ah;
            *reinterpret_cast<uint4*>(a_lo + off) = al;
            *reinterpret_cast<uint4*>(b_hi + off) = bh;
            *reinterpret_cast<uint4*>(b_lo + off) = bl;
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        // slice kt: hi product into columns 256 st + [0, 128), corrections into
        // 256 st + [128, 256), both started fresh
        const uint32_t t_hi = tmem + 256u * (uint32_t)st, t_co = t_hi + 128u;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int kk = 0; kk < BK; kk += 8) {
                const uint32_t off = (uint32_t)(kk >> 2) * LBO;
                const uint64_t dah = desc(smem_u32(a_hi) + off), dal = desc(smem_u32(a_lo) + off);
                const uint64_t dbh = desc(smem_u32(b_hi) + off), dbl = desc(smem_u32(b_lo) + off);
                mma_tf32(t_hi, dah, dbh, kk > 0 ? 1u : 0u);
                mma_tf32(t_co, dah, dbl, kk > 0 ? 1u : 0u);
                mma_tf32(t_co, dal, dbh, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar[st])));
        }
        // the global loads of slice kt+1 are in flight during the wait below
        if (kt + 1 < nkt) load_slice(kt + 1);
        // fold slice kt-1 into the registers while the tensor core runs slice kt
        // (the wait also frees stage kt-1's shared memory for slice kt+1)
        if (kt >= 1) {
            const int sp = st ^ 1;
            ok = __syncthreads_and(mbar_wait(smem_u32(&mbar[sp]), parity[sp]) ? 1 : 0) != 0;
            parity[sp] ^= 1u;
            if (!ok) {
                if (tid == 0) atomicOr(status, DEV_TC_TIMEOUT);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t p_hi = tmem + 256u * (uint32_t)sp + ((uint32_t)lane_base << 16) + (uint32_t)col_base;
#pragma unroll
            for (int c = 0; c < 64; c += 32) {
                uint32_t vh[32], vc[32];
                ld32<0>(p_hi + (uint32_t)c, vh);
                ld32<1>(p_hi + 128u + (uint32_t)c, vc);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[c + j] += __uint_as_float(vh[j]) + __uint_as_float(vc[j]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();  // accumulator pair sp is read: slice kt+1 may overwrite it
        }
    }
    // the last slice
    if (ok && nkt > 0) {
        const int sp = (nkt - 1) & 1;
        ok = __syncthreads_and(mbar_wait(smem_u32(&mbar[sp]), parity[sp]) ? 1 : 0) != 0;
        if (!ok) {
            if (tid == 0) atomicOr(status, DEV_TC_TIMEOUT);
        } else {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t p_hi = tmem + 256u * (uint32_t)sp + ((uint32_t)lane_base << 16) + (uint32_t)col_base;
#pragma unroll
            for (int c = 0; c < 64; c += 32) {
                uint32_t vh[32], vc[32];
                ld32<0>(p_hi + (uint32_t)c, vh);
                ld32<1>(p_hi + 128u + (uint32_t)c, vc);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[c + j] += __uint_as_float(vh[j]) + __uint_as_float(vc[j]);
            }
        }
    }
    if (ok) {
        const int m = m0 + lane_base + lane;
        if (m < M) {
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                const int n = n0 + col_base + j;
                if (n < N) sc(b, m, n, acc[j]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace thc
