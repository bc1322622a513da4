// gemm.cuh -- batched, shared-memory tiled SIMT GEMM with functor operands.
//
// C[b](m, n) = sum_k A[b](m, k) * B[b](k, n), with A and B produced element by
// element by loader functors (so the bond-2 MPO expansion, transposes and dtype
// conversions happen while a tile is staged into shared memory and never touch
// HBM) and C written by a store functor.  blockIdx.z is the batch index,
// blockIdx.y / blockIdx.x the row / column tile.
#pragma once

#include "common.cuh"

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
        for (int j = 0; j < TN; ++j) acc[i][j] = Acc(0);

    for (int k0 = 0; k0 < K; k0 += BK) {
        // A tile: consecutive threads walk k (row-major A is contiguous in k)
        for (int i = tid; i < BM * BK; i += NT) {
            const int mm = i / BK, kk = i % BK;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? Acc(la(b, m, k)) : Acc(0);
        }
        // B tile: consecutive threads walk n (row-major B is contiguous in n)
        for (int i = tid; i < BK * BN; i += NT) {
            const int kk = i / BN, nn = i % BN;
            const int k = k0 + kk, n = n0 + nn;
            Bs[kk][nn] = (k < K && n < N) ? Acc(lb(b, k, n)) : Acc(0);
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

// Launch helper: picks tile sizes per accumulator type.
template <class Acc, class LA, class LB, class SC>
inline cudaError_t launch_gemm(int batch, int M, int N, int K, const LA& la, const LB& lb,
                               const SC& sc, cudaStream_t st) {
    if (batch <= 0 || M <= 0 || N <= 0) return cudaSuccess;
    constexpr int BM = 64, BN = 64, TM = 4, TN = 4;
    constexpr int BK = sizeof(Acc) == 8 ? 8 : 16;
    dim3 grid(ceil_div(N, BN), ceil_div(M, BM), batch);
    k_gemm<Acc, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(M, N, K, la, lb, sc);
    return cudaGetLastError();
}

}  // namespace thc
