// Gram matrix G = Psi^T Psi of a plan's FP32 atoms, for the decode with
// Gram-updated correlations.  Not in the paper: from Eqs. 9 and 11,
//   <r - c psi_k, psi_m> = <r, psi_m> - c <psi_k, psi_m> = c_m - c G[k][m],
// so one MP step can update every correlation from one row of G.
//
// G[i][j] = sum_n psi_i[n] psi_j[n] over the zero-padded atom rows, each
// entry accumulated as one FP32 FMA chain in increasing n (so G is exactly
// symmetric: G[i][j] and G[j][i] multiply the same pairs in the same order).
// CUDA cores, 128 x 128 output tile per CTA, 8 x 8 per thread, 16-deep K
// slices staged transposed in shared memory.
#include <algorithm>

#include "mp_device.cuh"
#include "mp_internal.h"

namespace mpgb {

constexpr int kGT = 128;   // output tile
constexpr int kGK = 16;    // K slice

__global__ void __launch_bounds__(256) gram_matrix_kernel(const float* __restrict__ P, int M, int ldN,
                                                           float* __restrict__ G, int ldG) {
    __shared__ __align__(16) float As[kGK][kGT + 4];
    __shared__ __align__(16) float Bs[kGK][kGT + 4];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.y * kGT, j0 = blockIdx.x * kGT;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    // each thread stages 2 float4 of A and 2 of B per slice: row = q >> 2,
    // k offset = 4 (q & 3), for q = tid and tid + 256
    for (int k0 = 0; k0 < ldN; k0 += kGK) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = tid + 256 * h;
            const int row = q >> 2, kk = 4 * (q & 3);
            const int ia = i0 + row, jb = j0 + row;
            float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
            if (ia < M) va = __ldg(reinterpret_cast<const float4*>(P + static_cast<size_t>(ia) * ldN + k0 + kk));
            if (jb < M) vb = __ldg(reinterpret_cast<const float4*>(P + static_cast<size_t>(jb) * ldN + k0 + kk));
            As[kk + 0][row] = va.x;
            As[kk + 1][row] = va.y;
            As[kk + 2][row] = va.z;
            As[kk + 3][row] = va.w;
            Bs[kk + 0][row] = vb.x;
            Bs[kk + 1][row] = vb.y;
            Bs[kk + 2][row] = vb.z;
            Bs[kk + 3][row] = vb.w;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kGK; ++k) {
            float a[8], b[8];
            const float4 a0 = *reinterpret_cast<const float4*>(&As[k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[k][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[k][tx * 8]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[k][tx * 8 + 4]);
            a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
            a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
            b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
            b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int i = i0 + ty * 8 + u;
        if (i >= M) continue;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int j = j0 + tx * 8 + v;
            if (j < M) G[static_cast<size_t>(i) * ldG + j] = acc[u][v];
        }
    }
}

mp_status gram_prepare(PlanImpl* p, cudaStream_t st) {
    if (p->gram) return MP_OK;
    const int ldG = (p->M + 3) / 4 * 4;
    const size_t bytes = static_cast<size_t>(p->M) * ldG * sizeof(float);
    float* G = nullptr;
    cudaError_t e = cudaMalloc(&G, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(Gram matrix)");
    const dim3 grid((p->M + kGT - 1) / kGT, (p->M + kGT - 1) / kGT);
    gram_matrix_kernel<<<grid, 256, 0, st>>>(p->psi32, p->M, p->ldN, G, ldG);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(G);
        return cuda_fail(e, "Gram matrix");
    }
    p->launches++;
    p->gram = G;
    p->ldG = ldG;
    p->device_bytes += bytes;
    return MP_OK;
}

}  // namespace mpgb
