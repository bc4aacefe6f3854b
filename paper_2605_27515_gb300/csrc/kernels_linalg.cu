// Batched complex GEMM of the step whose shapes are read from device memory,
// templated on the real type (double for the FP64 form, float for FP32 parts).
//
// The step's GEMMs are small and their sizes change every step (bond dimensions
// live in device memory), while the launch configuration is fixed when the step is
// captured as a CUDA graph.  On this GPU one SM retires ~2 FP64 FMAs per clock, so
// a GEMM whose 32 x 32 output tiles cover only a few SMs runs at a few percent of
// the chip.  The kernel is therefore persistent over a fixed grid (two CTAs per SM
// when a workspace is given) and decides the decomposition at run time from the
// actual sizes: with T output tiles and G CTAs it splits the K range into
// s = min(G / T, ceil(K / 16), cap) parts, so that T * s work items keep the SMs
// busy.  Each (tile, part) item writes its partial tile to the workspace; the CTA
// that finishes a tile last (a per-tile counter, no waiting) adds the s partials in
// part order and applies alpha and beta, so the result does not depend on timing.

#include <algorithm>
#include <cfloat>
#include <type_traits>

#include "df64.cuh"
#include "qlb_internal.cuh"

namespace qlb {

namespace {

constexpr int GB_M = 32, GB_N = 32, GB_K = 16, G_THREADS = 256;
constexpr int GB_TILE = GB_M * GB_N;
constexpr int GB_SPLIT_CAP = 64;  // default cap on the K split

template <typename R>
__device__ __forceinline__ cx<R> ldop(const cx<R>* P, int op, long ld, int i, int k) {
  // element (i, k) of op(P)
  if (op == OP_N) return P[(long)i * ld + k];
  cx<R> v = P[(long)k * ld + i];
  if (op == OP_C) v.im = -v.im;
  return v;
}

// storage -> compute type of an operand, compute -> storage type of a result
template <typename C, typename S>
__device__ __forceinline__ cx<C> to_c(cx<S> v) {
  return mk<C>(C(v.re), C(v.im));
}
template <typename S, typename C>
__device__ __forceinline__ cx<S> to_s(cx<C> v) {
  return mk<S>((S)v.re, (S)v.im);
}
// a partial tile entry written by another CTA of this launch (past L1)
__device__ __forceinline__ cx<double> ldcg_cx(const cx<double>* p) { return mk<double>(__ldcg(&p->re), __ldcg(&p->im)); }
__device__ __forceinline__ cx<float> ldcg_cx(const cx<float>* p) { return mk<float>(__ldcg(&p->re), __ldcg(&p->im)); }
__device__ __forceinline__ cx<df64> ldcg_cx(const cx<df64>* p) {
  const float4 v = __ldcg((const float4*)p);
  return mk<df64>(df64(v.x, v.y), df64(v.z, v.w));
}
// acc += a * b
template <typename C>
__device__ __forceinline__ void cmac(cx<C>& acc, cx<C> a, cx<C> b) {
  cfma(acc, a, b);
}
template <>
__device__ __forceinline__ void cmac<df64>(cx<df64>& acc, cx<df64> a, cx<df64> b) {
  acc.re = df_mac(acc.re, a.re, b.re);
  acc.re = df_mac(acc.re, -a.im, b.im);
  acc.im = df_mac(acc.im, a.re, b.im);
  acc.im = df_mac(acc.im, a.im, b.re);
}

template <typename R>
__device__ __forceinline__ cx<R> gemm_alpha(const GemmDesc& g) {
  cx<R> alpha = mk<R>((R)g.alpha_re, (R)g.alpha_im);
  if (g.alpha_scale) {
    double s = *g.alpha_scale;
    if (g.alpha_scale_rsqrt) s = (s > 0.0) ? 1.0 / sqrt(s) : 0.0;
    alpha = cscale(alpha, (R)s);
  }
  return alpha;
}

// R: the storage type of A, B, C; Cm: the type the products are formed and summed in
// (R itself, or double-float for FP64 storage in the mixed forms)
template <typename R, typename Cm, bool GRP>
__global__ void __launch_bounds__(G_THREADS) k_gemm(const GemmDesc g_in, const int* __restrict__ d_in, double* prof,
                                                    const GemmDesc* __restrict__ grp) {
  // grouped launch: this CTA works on member blockIdx.y, whose descriptor (and dims)
  // come from the group's table (kept in shared memory, not registers); the K split
  // is decided on the member's nominal grid
  __shared__ GemmDesc s_g;
  if constexpr (GRP) {
    if (threadIdx.x == 0) s_g = grp[blockIdx.y];
    __syncthreads();
  }
  const GemmDesc& g = GRP ? s_g : g_in;
  const int* __restrict__ d = GRP ? s_g.dims : d_in;
  const int gnom = g.split_grid > 0 ? g.split_grid : (int)gridDim.x;
  const int m = dev_eval(g.m, d), n = dev_eval(g.n, d), K = dev_eval(g.k, d);
  const int nb1 = dev_eval(g.nb1, d), nb2 = dev_eval(g.nb2, d);
  const int nb = nb1 * nb2;
  if (m <= 0 || n <= 0 || nb <= 0) return;
  const int tm = (m + GB_M - 1) / GB_M, tn = (n + GB_N - 1) / GB_N;
  const long ntiles = (long)tm * tn * nb;
  // the K split of this launch, from the run-time sizes (the same in every CTA)
  int ks = 1;
  if (g.ws && K > GB_K && ntiles < (long)gnom) {
    const int cap = g.ksplit >= 1 ? g.ksplit : GB_SPLIT_CAP;
    ks = (int)min((long)cap, (long)gnom / ntiles);
    ks = min(ks, (K + GB_K - 1) / GB_K);
    if (ks < 1) ks = 1;
  }
  const int chunk = ks > 1 ? (((K + ks - 1) / ks + GB_K - 1) / GB_K) * GB_K : K;
  if (ks > 1) ks = (K + chunk - 1) / chunk;
  if (prof && blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAdd(prof, 8.0 * (double)m * (double)n * (double)K * nb);
    atomicAdd(prof + QLB_K_COUNT, (double)sizeof(cx<R>) * ((double)m * K + (double)K * n + (double)m * n) * nb);
  }
  const long lda = dev_eval(g.lda, d), ldb = dev_eval(g.ldb, d), ldc = dev_eval(g.ldc, d);
  cx<Cm>* part_ws = (cx<Cm>*)g.ws;
  int* counters = g.ws ? (int*)(part_ws + (long)gnom * GB_TILE) : nullptr;

  __shared__ cx<Cm> As[GB_K][GB_M + 1];
  __shared__ cx<Cm> Bs[GB_K][GB_N + 1];
  __shared__ int s_last;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const long items = ntiles * ks;
  for (long it = blockIdx.x; it < items; it += gridDim.x) {
    const long tile = it / ks;
    const int kp = (int)(it - tile * ks);
    const int bz = (int)(tile / ((long)tm * tn));
    const int t2 = (int)(tile - (long)bz * tm * tn);
    const int row0 = (t2 / tn) * GB_M, col0 = (t2 % tn) * GB_N;
    const int b1 = bz / nb2, b2 = bz - b1 * nb2;
    const cx<R>* A = (const cx<R>*)g.A + (long)b1 * dev_eval(g.sA1, d) + (long)b2 * dev_eval(g.sA2, d);
    const cx<R>* B = (const cx<R>*)g.B + (long)b1 * dev_eval(g.sB1, d) + (long)b2 * dev_eval(g.sB2, d);
    cx<R>* C = (cx<R>*)g.C + (long)b1 * dev_eval(g.sC1, d) + (long)b2 * dev_eval(g.sC2, d);
    const int kbeg = kp * chunk, kend = min(K, kbeg + chunk);

    // warp-uniform: does this warp own an output row of the tile (rows 2w, 2w + 1
    // of each half), and does the tile reach the upper column half
    const int wrow = row0 + 2 * (tid >> 5);
    const bool do_r0 = wrow < m, do_r1 = wrow + 16 < m, do_c1 = col0 + 16 < n;
    cx<Cm> acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
      for (int j = 0; j < 2; j++) acc[i][j] = to_c<Cm>(mk<R>(0, 0));
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
        As[kk][i] = to_c<Cm>((gi < m && gk < kend) ? ldop(A, g.opA, lda, gi, gk) : mk<R>(0, 0));
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
        Bs[kk][j] = to_c<Cm>(v);
      }
      __syncthreads();
      // the products of the padding are skipped where a whole warp would form only
      // padding (warp-uniform tests: the warp's rows, the upper column half, the
      // K tail), which on the slow FP64 pipe is most of the work of a small GEMM
      const int kn = min(GB_K, kend - k0);
      if (kn == GB_K && do_r1 && do_c1) {
#pragma unroll
        for (int kk = 0; kk < GB_K; kk++) {
          cx<Cm> a0 = As[kk][ty], a1 = As[kk][ty + 16];
          cx<Cm> b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
          cmac(acc[0][0], a0, b0);
          cmac(acc[0][1], a0, b1);
          cmac(acc[1][0], a1, b0);
          cmac(acc[1][1], a1, b1);
        }
      } else if (do_r0) {
#pragma unroll 4
        for (int kk = 0; kk < kn; kk++) {
          cx<Cm> a0 = As[kk][ty];
          cx<Cm> b0 = Bs[kk][tx];
          cmac(acc[0][0], a0, b0);
          if (do_c1) cmac(acc[0][1], a0, Bs[kk][tx + 16]);
          if (do_r1) {
            cx<Cm> a1 = As[kk][ty + 16];
            cmac(acc[1][0], a1, b0);
            if (do_c1) cmac(acc[1][1], a1, Bs[kk][tx + 16]);
          }
        }
      }
      __syncthreads();
    }
    if (ks > 1) {
      // partial tile of this K part; the last CTA of the tile adds them in order
      cx<Cm>* P = part_ws + ((long)kp * ntiles + tile) * GB_TILE;
      // (only the entries inside the output are written and read back)
#pragma unroll
      for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++)
          if (row0 + ty + 16 * i < m && col0 + tx + 16 * j < n) P[(ty + 16 * i) * GB_N + tx + 16 * j] = acc[i][j];
      __threadfence();
      __syncthreads();
      if (tid == 0) s_last = atomicAdd(counters + tile, 1) == ks - 1;
      __syncthreads();
      if (!s_last) continue;
      __threadfence();
#pragma unroll
      for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) {
          if (row0 + ty + 16 * i >= m || col0 + tx + 16 * j >= n) continue;
          cx<Cm> sum = to_c<Cm>(mk<R>(0, 0));
          const long off = (long)(ty + 16 * i) * GB_N + tx + 16 * j;
          const long pstride = ntiles * GB_TILE;
          const cx<Cm>* P0 = part_ws + tile * GB_TILE + off;
          int s = 0;
          // four independent loads in flight, added in part order
          for (; s + 4 <= ks; s += 4) {
            const cx<Cm> v0 = ldcg_cx(P0 + s * pstride), v1 = ldcg_cx(P0 + (s + 1) * pstride);
            const cx<Cm> v2 = ldcg_cx(P0 + (s + 2) * pstride), v3 = ldcg_cx(P0 + (s + 3) * pstride);
            sum = cadd(cadd(cadd(cadd(sum, v0), v1), v2), v3);
          }
          for (; s < ks; s++) sum = cadd(sum, ldcg_cx(P0 + s * pstride));
          acc[i][j] = sum;
        }
      if (tid == 0) counters[tile] = 0;  // ready for the next launch on this workspace
    }
    const cx<R> alpha = gemm_alpha<R>(g);
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
      for (int j = 0; j < 2; j++) {
        int gi = row0 + ty + 16 * i, gj = col0 + tx + 16 * j;
        if (gi < m && gj < n) {
          cx<R> v = cmul(alpha, to_s<R>(acc[i][j]));
          cx<R>* dst = C + (long)gi * ldc + gj;
          if (g.beta) v = cadd(v, *dst);
          *dst = v;
        }
      }
  }
}

}  // namespace

size_t gemm_workspace_elems(int grid) {
  // grid partial tiles, then one counter (int) per tile, rounded up to whole elements
  return (size_t)grid * GB_TILE + ((size_t)grid * sizeof(int) + sizeof(zd) - 1) / sizeof(zd);
}

int gemm_grid_default() {
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
      cudaGetLastError();
      sms = 148;
    }
    grid = 2 * sms;
  }
  return grid;
}

template <typename R>
cudaError_t launch_gemm(const GemmDesc& g, const int* d_dims, cudaStream_t s, double* prof) {
  const long planned = (long)((g.m_max + GB_M - 1) / GB_M) * ((g.n_max + GB_N - 1) / GB_N) *
                       (g.nb_max > 0 ? g.nb_max : 1);
  if (planned <= 0) return cudaSuccess;
  // with a workspace: a fixed grid that the run-time split fills; without: one CTA
  // per planned tile (persistent above 4096)
  const int grid = g.ws ? (g.grid > 0 ? g.grid : gemm_grid_default()) : (int)std::min<long>(planned, 4096);
  GemmDesc gg = g;
  if (!g.ws) gg.ksplit = 1;
  gg.split_grid = 0;
  if constexpr (std::is_same<R, double>::value) {
    if (g.df64) {
      k_gemm<R, df64, false><<<grid, G_THREADS, 0, s>>>(gg, d_dims, prof, nullptr);
      return cudaGetLastError();
    }
  }
  k_gemm<R, R, false><<<grid, G_THREADS, 0, s>>>(gg, d_dims, prof, nullptr);
  return cudaGetLastError();
}

template cudaError_t launch_gemm<double>(const GemmDesc&, const int*, cudaStream_t, double*);
template cudaError_t launch_gemm<float>(const GemmDesc&, const int*, cudaStream_t, double*);

// The same GEMM of S states in one launch: grid (per-member CTAs, S).  Every member
// descriptor in d_grp carries its dims, a workspace for the default grid and
// split_grid = the default grid, so each member is split and summed exactly as in
// its own launch; the per-member CTA count only changes how the work items are
// shared out (S x per-member CTAs ~ two per SM over the whole group).
cudaError_t launch_gemm_group(const GemmDesc* d_grp, int S, int use_df, cudaStream_t s, double* prof) {
  if (S <= 0) return cudaSuccess;
  const int full = gemm_grid_default();
  const int per = std::max(8, std::min(full, (full + S - 1) / S));
  GemmDesc dummy{};
  if (use_df)
    k_gemm<double, df64, true><<<dim3(per, S), G_THREADS, 0, s>>>(dummy, nullptr, prof, d_grp);
  else
    k_gemm<double, double, true><<<dim3(per, S), G_THREADS, 0, s>>>(dummy, nullptr, prof, d_grp);
  return cudaGetLastError();
}

}  // namespace qlb
