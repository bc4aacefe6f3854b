// Batched complex GEMM of the step whose shapes are read from device memory,
// templated on the real type (double for the FP64 form, float for FP32 parts).

#include <algorithm>
#include <cfloat>

#include "qlb_internal.cuh"

namespace qlb {

// =====================================================================================
// batched complex GEMM, shapes from device memory
// =====================================================================================

namespace {

constexpr int GB_M = 32, GB_N = 32, GB_K = 16, G_THREADS = 256;

template <typename R>
__device__ __forceinline__ cx<R> ldop(const cx<R>* P, int op, long ld, int i, int k) {
  // element (i, k) of op(P)
  if (op == OP_N) return P[(long)i * ld + k];
  cx<R> v = P[(long)k * ld + i];
  if (op == OP_C) v.im = -v.im;
  return v;
}

template <typename R>
__global__ void __launch_bounds__(G_THREADS) k_gemm(GemmDesc g, const int* __restrict__ d, double* prof) {
  const int m = dev_eval(g.m, d), n = dev_eval(g.n, d), K = dev_eval(g.k, d);
  const int nb1 = dev_eval(g.nb1, d), nb2 = dev_eval(g.nb2, d);
  const int nsplit = g.ksplit > 1 ? g.ksplit : 1;
  const int bz = blockIdx.z / nsplit, ks = blockIdx.z - (blockIdx.z / nsplit) * nsplit;
  if (bz >= nb1 * nb2 || m <= 0 || n <= 0) return;
  const int row0 = blockIdx.y * GB_M, col0 = blockIdx.x * GB_N;
  if (row0 >= m || col0 >= n) return;
  const int b1 = bz / nb2, b2 = bz - b1 * nb2;
  const long lda = dev_eval(g.lda, d), ldb = dev_eval(g.ldb, d), ldc = dev_eval(g.ldc, d);
  const cx<R>* A = (const cx<R>*)g.A + (long)b1 * dev_eval(g.sA1, d) + (long)b2 * dev_eval(g.sA2, d);
  const cx<R>* B = (const cx<R>*)g.B + (long)b1 * dev_eval(g.sB1, d) + (long)b2 * dev_eval(g.sB2, d);
  cx<R>* C = (cx<R>*)g.C + (long)b1 * dev_eval(g.sC1, d) + (long)b2 * dev_eval(g.sC2, d);

  // K range of this CTA (the whole range without split-K)
  int kbeg = 0, kend = K;
  if (nsplit > 1) {
    const int chunk = (((K + nsplit - 1) / nsplit) + GB_K - 1) / GB_K * GB_K;
    kbeg = min(K, ks * chunk);
    kend = min(K, kbeg + chunk);
  }
  if (prof && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) {
    double nb = (double)(nb1 * nb2);
    atomicAdd(prof, 8.0 * (double)m * (double)n * (double)K * nb);
    atomicAdd(prof + QLB_K_COUNT, (double)sizeof(cx<R>) * ((double)m * K + (double)K * n + (double)m * n) * nb);
  }

  __shared__ cx<R> As[GB_K][GB_M + 1];
  __shared__ cx<R> Bs[GB_K][GB_N + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  cx<R> acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 2; j++) acc[i][j] = mk<R>(0, 0);

  for (int k0 = kbeg; k0 < kend; k0 += GB_K) {
    // A tile: rows row0.., cols k0..
    for (int e = tid; e < GB_M * GB_K; e += G_THREADS) {
      int i, kk;
      if (g.opA == OP_N) {
        kk = e % GB_K;
        i = e / GB_K;
      } else {
        i = e % GB_M;
        kk = e / GB_M;
      }
      int gi = row0 + i, gk = k0 + kk;
      As[kk][i] = (gi < m && gk < kend) ? ldop(A, g.opA, lda, gi, gk) : mk<R>(0, 0);
    }
    for (int e = tid; e < GB_N * GB_K; e += G_THREADS) {
      int j, kk;
      if (g.opB == OP_N) {
        j = e % GB_N;
        kk = e / GB_N;
      } else {
        kk = e % GB_K;
        j = e / GB_K;
      }
      int gj = col0 + j, gk = k0 + kk;
      // op(B)(k, j): OP_N B[k*ldb + j]; OP_T B[j*ldb + k]
      cx<R> v = mk<R>(0, 0);
      if (gj < n && gk < kend) {
        if (g.opB == OP_N)
          v = B[(long)gk * ldb + gj];
        else {
          v = B[(long)gj * ldb + gk];
          if (g.opB == OP_C) v.im = -v.im;
        }
      }
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GB_K; kk++) {
      cx<R> a0 = As[kk][ty], a1 = As[kk][ty + 16];
      cx<R> b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      cfma(acc[0][0], a0, b0);
      cfma(acc[0][1], a0, b1);
      cfma(acc[1][0], a1, b0);
      cfma(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
  if (nsplit > 1) {
    // partial sums of this K range; the reduction applies alpha and beta
    cx<R>* W = (cx<R>*)g.ws + ((long)ks * g.nb_max + bz) * (long)g.m_max * g.n_max;
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
      for (int j = 0; j < 2; j++) {
        int gi = row0 + ty + 16 * i, gj = col0 + tx + 16 * j;
        if (gi < m && gj < n) W[(long)gi * g.n_max + gj] = acc[i][j];
      }
    return;
  }
  cx<R> alpha = mk<R>((R)g.alpha_re, (R)g.alpha_im);
  if (g.alpha_scale) {
    double s = *g.alpha_scale;
    if (g.alpha_scale_rsqrt) s = (s > 0.0) ? 1.0 / sqrt(s) : 0.0;
    alpha = cscale(alpha, (R)s);
  }
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 2; j++) {
      int gi = row0 + ty + 16 * i, gj = col0 + tx + 16 * j;
      if (gi < m && gj < n) {
        cx<R> v = cmul(alpha, acc[i][j]);
        cx<R>* dst = C + (long)gi * ldc + gj;
        if (g.beta) v = cadd(v, *dst);
        *dst = v;
      }
    }
}

// C = alpha * sum_s W[s] (+ C): the split-K partial sums added in split order.
template <typename R>
__global__ void k_gemm_splitk_sum(GemmDesc g, const int* __restrict__ d) {
  const int m = dev_eval(g.m, d), n = dev_eval(g.n, d);
  const int nb1 = dev_eval(g.nb1, d), nb2 = dev_eval(g.nb2, d);
  const long ldc = dev_eval(g.ldc, d);
  cx<R> alpha = mk<R>((R)g.alpha_re, (R)g.alpha_im);
  if (g.alpha_scale) {
    double s = *g.alpha_scale;
    if (g.alpha_scale_rsqrt) s = (s > 0.0) ? 1.0 / sqrt(s) : 0.0;
    alpha = cscale(alpha, (R)s);
  }
  const long per = (long)m * n, total = per * nb1 * nb2;
  const long slab = (long)g.m_max * g.n_max;
  for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < total; x += (long)gridDim.x * blockDim.x) {
    const int bz = (int)(x / per);
    const long r = x - (long)bz * per;
    const int i = (int)(r / n), j = (int)(r - (long)i * n);
    const int b1 = bz / nb2, b2 = bz - b1 * nb2;
    cx<R> acc = mk<R>(0, 0);
    for (int s = 0; s < g.ksplit; s++) acc = cadd(acc, ((const cx<R>*)g.ws)[((long)s * g.nb_max + bz) * slab + (long)i * g.n_max + j]);
    cx<R>* C = (cx<R>*)g.C + (long)b1 * dev_eval(g.sC1, d) + (long)b2 * dev_eval(g.sC2, d);
    cx<R> v = cmul(alpha, acc);
    if (g.beta) v = cadd(v, C[(long)i * ldc + j]);
    C[(long)i * ldc + j] = v;
  }
}

}  // namespace

template <typename R>
cudaError_t launch_gemm(const GemmDesc& g, const int* d_dims, cudaStream_t s, double* prof) {
  const int nsplit = g.ksplit > 1 && g.ws ? g.ksplit : 1;
  GemmDesc gg = g;
  gg.ksplit = nsplit;
  const int nb = g.nb_max > 0 ? g.nb_max : 1;
  dim3 grid((g.n_max + GB_N - 1) / GB_N, (g.m_max + GB_M - 1) / GB_M, nb * nsplit);
  if (grid.x == 0 || grid.y == 0) return cudaSuccess;
  k_gemm<R><<<grid, G_THREADS, 0, s>>>(gg, d_dims, prof);
  if (nsplit > 1) {
    long total = (long)g.m_max * g.n_max * nb;
    unsigned blocks = (unsigned)std::min<long>(4 * 152, (total + 255) / 256);
    k_gemm_splitk_sum<R><<<blocks, 256, 0, s>>>(gg, d_dims);
  }
  return cudaGetLastError();
}

template cudaError_t launch_gemm<double>(const GemmDesc&, const int*, cudaStream_t, double*);
template cudaError_t launch_gemm<float>(const GemmDesc&, const int*, cudaStream_t, double*);

}  // namespace qlb
