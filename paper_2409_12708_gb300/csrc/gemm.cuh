// gemm.cuh -- batched, shared-memory tiled SIMT GEMM with functor operands
// (real or complex accumulators).
//
// C[b](m, n) = sum_k A[b](m, k) * B[b](k, n), with A and B produced element by
// element by loader functors (so the bond-2 MPO expansion, transposes and dtype
// conversions happen while a tile is staged into shared memory and never touch
// HBM) and C written by a store functor.  blockIdx.z is the batch index,
// blockIdx.y / blockIdx.x the row / column tile.
#pragma once

#include "common.cuh"
#include "scalar.cuh"

namespace thc {

template <class Acc, int BM, int BN, int BK, int TM, int TN, class LA, class LB, class SC>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm(int M, int N, int K, LA la, LB lb, SC sc) {
    constexpr int TX = BN / TN;          // threads along n
    constexpr int TY = BM / TM;          // threads along m
    constexpr int NT = TX * TY;
    __shared__ Acc As[BK][BM + 1];
    __shared__ Acc Bs[BK][BN + 1];
    const int b = blockIdx.z;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    Acc acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = tzero<Acc>();

    for (int k0 = 0; k0 < K; k0 += BK) {
        // A tile: consecutive threads walk k (row-major A is contiguous in k)
        for (int i = tid; i < BM * BK; i += NT) {
            const int mm = i / BK, kk = i % BK;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? cvt<Acc>(la(b, m, k)) : tzero<Acc>();
        }
        // B tile: consecutive threads walk n (row-major B is contiguous in n)
        for (int i = tid; i < BK * BN; i += NT) {
            const int kk = i / BN, nn = i % BN;
            const int k = k0 + kk, n = n0 + nn;
            Bs[kk][nn] = (k < K && n < N) ? cvt<Acc>(lb(b, k, n)) : tzero<Acc>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            Acc av[TM], bv[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) av[i] = As[kk][ty + i * TY];
#pragma unroll
            for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + j * TX];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int m = m0 + ty + i * TY;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int n = n0 + tx + j * TX;
            if (n < N) sc(b, m, n, acc[i][j]);
        }
    }
}

// Large-tile float32 variant: 128 x 128 tile, 256 threads, each thread an 8 x 8
// block of C made of four 4 x 4 quadrants (rows 4ty.. and 64+4ty.., columns
// 4tx.. and 64+4tx..), so every k step reads its operands with four 16-byte
// shared-memory loads for 64 FMAs.
template <int BK, class LA, class LB, class SC>
__global__ void __launch_bounds__(256) k_gemm128(int M, int N, int K, LA la, LB lb, SC sc) {
    constexpr int BM = 128, BN = 128, LDS = BM + 4;
    __shared__ __align__(16) float As[BK][LDS];
    __shared__ __align__(16) float Bs[BK][LDS];
    const int b = blockIdx.z;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int i = tid; i < BM * BK; i += 256) {
            const int mm = i / BK, kk = i % BK;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? float(la(b, m, k)) : 0.f;
        }
        for (int i = tid; i < BK * BN; i += 256) {
            const int kk = i / BN, nn = i % BN;
            const int k = k0 + kk, n = n0 + nn;
            Bs[kk][nn] = (k < K && n < N) ? float(lb(b, k, n)) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][4 * ty]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][64 + 4 * ty]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][4 * tx]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][64 + 4 * tx]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + i - 4);
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = n0 + (j < 4 ? 4 * tx + j : 64 + 4 * tx + j - 4);
            if (n < N) sc(b, m, n, acc[i][j]);
        }
    }
}

// Launch helper: picks tile sizes per accumulator type (the large-tile float32
// kernel when both output dimensions fill its tile).
template <class Acc, class LA, class LB, class SC>
inline cudaError_t launch_gemm(int batch, int M, int N, int K, const LA& la, const LB& lb,
                               const SC& sc, cudaStream_t st) {
    if (batch <= 0 || M <= 0 || N <= 0) return cudaSuccess;
    if constexpr (sizeof(Acc) == 4) {
        if (M >= 128 && N >= 128) {
            dim3 grid(ceil_div(N, 128), ceil_div(M, 128), batch);
            k_gemm128<16><<<grid, 256, 0, st>>>(M, N, K, la, lb, sc);
            return cudaGetLastError();
        }
    }
    constexpr int BM = 64, BN = 64, TM = 4, TN = 4;
    constexpr int BK = sizeof(Acc) >= 8 ? 8 : 16;
    dim3 grid(ceil_div(N, BN), ceil_div(M, BM), batch);
    k_gemm<Acc, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(M, N, K, la, lb, sc);
    return cudaGetLastError();
}

}  // namespace thc
