// Dense complex linear algebra of the step: a batched GEMM whose shapes are read
// from device memory, and a one-CTA cyclic Jacobi Hermitian eigensolver that
// ends with the truncation decision of the bond it serves.
//
// Both are templated on the real type (double for the FP64 form, float for the
// FP32 parts of the mixed form).

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
  const int bz = blockIdx.z;
  if (bz >= nb1 * nb2 || m <= 0 || n <= 0) return;
  const int row0 = blockIdx.y * GB_M, col0 = blockIdx.x * GB_N;
  if (row0 >= m || col0 >= n) return;
  const int b1 = bz / nb2, b2 = bz - b1 * nb2;
  const long lda = dev_eval(g.lda, d), ldb = dev_eval(g.ldb, d), ldc = dev_eval(g.ldc, d);
  const cx<R>* A = (const cx<R>*)g.A + (long)b1 * dev_eval(g.sA1, d) + (long)b2 * dev_eval(g.sA2, d);
  const cx<R>* B = (const cx<R>*)g.B + (long)b1 * dev_eval(g.sB1, d) + (long)b2 * dev_eval(g.sB2, d);
  cx<R>* C = (cx<R>*)g.C + (long)b1 * dev_eval(g.sC1, d) + (long)b2 * dev_eval(g.sC2, d);

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

  for (int k0 = 0; k0 < K; k0 += GB_K) {
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
      As[kk][i] = (gi < m && gk < K) ? ldop(A, g.opA, lda, gi, gk) : mk<R>(0, 0);
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
      if (gj < n && gk < K) {
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

}  // namespace

template <typename R>
cudaError_t launch_gemm(const GemmDesc& g, const int* d_dims, cudaStream_t s, double* prof) {
  dim3 grid((g.n_max + GB_N - 1) / GB_N, (g.m_max + GB_M - 1) / GB_M, g.nb_max > 0 ? g.nb_max : 1);
  if (grid.x == 0 || grid.y == 0) return cudaSuccess;
  k_gemm<R><<<grid, G_THREADS, 0, s>>>(g, d_dims, prof);
  return cudaGetLastError();
}

template cudaError_t launch_gemm<double>(const GemmDesc&, const int*, cudaStream_t, double*);
template cudaError_t launch_gemm<float>(const GemmDesc&, const int*, cudaStream_t, double*);

// =====================================================================================
// one-CTA cyclic Jacobi for a Hermitian matrix, with the truncation decision
// =====================================================================================
//
// Parallel (round-robin) ordering: in each of the np-1 rounds of a sweep the np
// indices form np/2 disjoint pairs, all rotated at once.  The rotation of pair
// (p, q) is J = [[c, sp], [-conj(sp), c]] with sp = s e^{i phi}, phi = arg G[p,q]
// and (c, s) the real symmetric Schur pair of [[G_pp, |G_pq|], [|G_pq|, G_qq]]
// (Golub & Van Loan, sym.schur2); G <- J^dag G J, V <- V J.  A pair is skipped
// when |G_pq| <= n eps sqrt(|G_pp G_qq|) (the relative criterion that keeps small
// eigenvalues of a Gram matrix accurate) or below an absolute floor of
// eps Tr G; a sweep with no rotation ends the solve.

namespace {

constexpr int E_THREADS = 512;

template <typename R>
struct Eps;
template <>
struct Eps<double> {
  static constexpr double v = 2.220446049250313e-16;
};
template <>
struct Eps<float> {
  static constexpr float v = 1.1920929e-07f;
};

__device__ __forceinline__ int rr_player(int pos, int round, int np) {
  if (pos == 0) return 0;
  return 1 + (pos - 1 + round) % (np - 1);
}

// The truncation rule (relative discarded weight, cap, degeneracy clusters);
// w[] sorted descending, non-negative.  Returns k >= 1.
__device__ int keep_count_dev(const double* w, int n, double tol, int cap, double gap) {
  if (n <= 0) return 0;
  double total = 0.0;
  for (int i = 0; i < n; i++) total += w[i];
  if (!(total > 0.0)) return 1;
  int k = n;
  double tail = 0.0;
  while (k > 1 && tail + w[k - 1] <= tol * total) {
    tail += w[k - 1];
    k--;
  }
  if (k > cap) k = cap;
  if (k < 1) k = 1;
  if (k < n) {
    double sk = sqrt(w[k]), skm = sqrt(w[k - 1]);
    if (sk >= (1.0 - gap) * skm) {
      int j = k;
      while (j < n && j < cap && sqrt(w[j]) >= (1.0 - gap) * sqrt(w[j - 1])) j++;
      if (j < n && sqrt(w[j]) >= (1.0 - gap) * sqrt(w[j - 1])) {
        j = k;
        while (j > 1 && sqrt(w[j]) >= (1.0 - gap) * sqrt(w[j - 1])) j--;
      }
      k = j;
    }
  }
  return k < 1 ? 1 : k;
}

template <typename R>
__global__ void __launch_bounds__(E_THREADS) k_eig(EigDesc e, int* __restrict__ d, cx<R>* work, int use_smem,
                                                  double* prof) {
  extern __shared__ unsigned char smem_raw[];
  const int n = dev_eval(e.n, d);
  const int tid = threadIdx.x;
  if (n <= 0) {
    if (tid == 0) d[e.dim_out] = 0;
    return;
  }
  const int np = n + (n & 1);
  cx<R>* Gs;
  cx<R>* Vs;
  if (use_smem) {
    Gs = (cx<R>*)smem_raw;
    Vs = Gs + (long)np * np;
  } else {
    Gs = work;
    Vs = work + (long)np * np;
  }
  __shared__ R rc[256];
  __shared__ cx<R> rsp[256];
  __shared__ int rp[256], rq[256];
  __shared__ int n_rot;
  __shared__ int s_perm[512];
  __shared__ double s_w[512];
  __shared__ int s_k;
  __shared__ int s_bad;
  __shared__ R s_thr;
  __shared__ double s_tr;
  __shared__ double s_off;

  const cx<R>* G = (const cx<R>*)e.G;
  for (long x = tid; x < (long)np * np; x += E_THREADS) {
    int i = (int)(x / np), j = (int)(x - (long)i * np);
    cx<R> v = mk<R>(0, 0);
    if (i < n && j < n) v = G[(long)i * n + j];
    if (i == j) v.im = 0;
    Gs[x] = v;
    Vs[x] = mk<R>(i == j ? (R)1 : (R)0, (R)0);
  }
  if (tid == 0) {
    s_bad = 0;
    double tr = 0;
    for (int i = 0; i < n; i++) tr += fabs((double)Gs[(long)i * np + i].re);
    // absolute floor 2 eps^2 Tr G: couplings below it change no eigenvalue above
    // eps^2 Tr G.  Noise among the null directions of a rank-deficient Gram matrix
    // can keep rotating above it; the solve then stops at the sweep limit and is
    // accepted when the off-diagonal norm left is below n eps Tr G (its rounding).
    s_thr = (R)((double)Eps<R>::v * (double)Eps<R>::v * 2.0 * tr);
    s_tr = tr;
  }
  __syncthreads();
  const R abs_thr = s_thr;
  // relative floor: rounding in the row/column updates leaves off-diagonals of
  // order n eps sqrt(G_pp G_qq); asking for less would rotate noise forever
  const R rel_tol = Eps<R>::v * (R)(n > 8 ? n : 8);

  const int npairs = np / 2;
  int sweep = 0;
  long total_rot = 0;
  for (; sweep < e.max_sweeps; sweep++) {
    if (tid == 0) n_rot = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; round++) {
      if (tid < npairs) {
        int p = rr_player(tid, round, np), q = rr_player(np - 1 - tid, round, np);
        if (p > q) {
          int t = p;
          p = q;
          q = t;
        }
        R c = 1, s = 0;
        cx<R> sp = mk<R>(0, 0);
        bool rot = false;
        if (q < n) {
          R a = Gs[(long)p * np + p].re, b = Gs[(long)q * np + q].re;
          cx<R> gpq = Gs[(long)p * np + q];
          R x = sqrt(cabs2(gpq));
          if (x > rel_tol * sqrt(fabs(a * b)) && x > abs_thr && x > (R)0) {
            R tau = (b - a) / (2 * x);
            R t = fabs(tau) > (R)1e15 ? (R)0.5 / tau : (tau >= 0 ? (R)1 : (R)-1) / (fabs(tau) + sqrt((R)1 + tau * tau));
            c = (R)1 / sqrt((R)1 + t * t);
            s = t * c;
            sp = mk<R>(s * gpq.re / x, s * gpq.im / x);
            rot = true;
          }
        }
        rc[tid] = c;
        rsp[tid] = sp;
        rp[tid] = rot ? p : -1;
        rq[tid] = q;
        if (rot) atomicAdd(&n_rot, 1);
      }
      __syncthreads();
      // rows: G <- J^dag G
      for (int w = tid; w < npairs * np; w += E_THREADS) {
        int t = w / np, j = w - t * np;
        int p = rp[t];
        if (p < 0) continue;
        int q = rq[t];
        R c = rc[t];
        cx<R> sp = rsp[t];
        cx<R> gp = Gs[(long)p * np + j], gq = Gs[(long)q * np + j];
        cx<R> np_ = csub(cscale(gp, c), cmul(sp, gq));
        cx<R> nq_ = cadd(cmul(cconj(sp), gp), cscale(gq, c));
        Gs[(long)p * np + j] = np_;
        Gs[(long)q * np + j] = nq_;
      }
      __syncthreads();
      // columns: G <- G J, V <- V J
      for (int w = tid; w < npairs * np; w += E_THREADS) {
        int t = w / np, i = w - t * np;
        int p = rp[t];
        if (p < 0) continue;
        int q = rq[t];
        R c = rc[t];
        cx<R> sp = rsp[t];
        cx<R> gp = Gs[(long)i * np + p], gq = Gs[(long)i * np + q];
        Gs[(long)i * np + p] = csub(cscale(gp, c), cmul(cconj(sp), gq));
        Gs[(long)i * np + q] = cadd(cmul(sp, gp), cscale(gq, c));
        cx<R> vp = Vs[(long)i * np + p], vq = Vs[(long)i * np + q];
        Vs[(long)i * np + p] = csub(cscale(vp, c), cmul(cconj(sp), vq));
        Vs[(long)i * np + q] = cadd(cmul(sp, vp), cscale(vq, c));
      }
      __syncthreads();
      // the rotated pairs' off-diagonal entries are zero by construction
      if (tid < npairs && rp[tid] >= 0) {
        int p = rp[tid], q = rq[tid];
        Gs[(long)p * np + q] = mk<R>(0, 0);
        Gs[(long)q * np + p] = mk<R>(0, 0);
        Gs[(long)p * np + p].im = 0;
        Gs[(long)q * np + q].im = 0;
      }
      __syncthreads();
    }
    int nr = n_rot;
    total_rot += nr;
    __syncthreads();
    if (nr == 0) break;
  }
  bool unconverged = false;
  if (sweep >= e.max_sweeps) {
    // accept a solve whose remaining couplings are at the rounding level
    if (tid == 0) s_off = 0.0;
    __syncthreads();
    double acc = 0.0;
    for (long x = tid; x < (long)n * n; x += E_THREADS) {
      int i = (int)(x / n), j = (int)(x - (long)i * n);
      if (i != j) acc += (double)cabs2(Gs[(long)i * np + j]);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) atomicAdd(&s_off, acc);
    __syncthreads();
    double lim = (double)n * (double)Eps<R>::v * s_tr;
    unconverged = !(sqrt(s_off) <= lim);
  }
  if (prof && tid == 0) {
    atomicAdd(prof, 60.0 * (double)np * (double)total_rot);
    atomicAdd(prof + QLB_K_COUNT, 2.0 * sizeof(cx<R>) * (double)n * (double)n);
  }

  // eigenvalues, sorted descending (stable on index)
  for (int i = tid; i < n; i += E_THREADS) {
    double li = (double)Gs[(long)i * np + i].re;
    if (!isfinite(li)) s_bad = 1;
    int rank = 0;
    for (int j = 0; j < n; j++) {
      double lj = (double)Gs[(long)j * np + j].re;
      if (lj > li || (lj == li && j < i)) rank++;
    }
    s_perm[rank] = i;
  }
  __syncthreads();
  for (int r = tid; r < n; r += E_THREADS) {
    double l = (double)Gs[(long)s_perm[r] * np + s_perm[r]].re;
    s_w[r] = l > 0.0 ? l : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    int cap = dev_eval(e.cap, d);
    if (cap < 1) cap = 1;
    int k = s_bad ? 1 : keep_count_dev(s_w, n, e.tol, cap, e.gap);
    s_k = k;
    d[e.dim_out] = k;
    double total = 0.0, kept = 0.0;
    for (int i = 0; i < n; i++) total += s_w[i];
    for (int i = 0; i < k; i++) kept += s_w[i];
    if (e.kept_weight) *e.kept_weight = kept;
    if (e.total_weight) *e.total_weight = total;
    if (e.disc_stat && total > 0.0) {
      double r = (total - kept) / total;
      if (r > *e.disc_stat) *e.disc_stat = r;
    }
    if (e.lam)
      for (int i = 0; i < n; i++) e.lam[i] = s_w[i];
    if (e.err) {
      if (unconverged) atomicOr(e.err, 1);
      if (s_bad || !isfinite(total)) atomicOr(e.err, 2);
    }
  }
  __syncthreads();
  const int k = s_k;
  cx<R>* out = (cx<R>*)e.out;
  if (e.out_mode == 0) {
    for (long x = tid; x < (long)n * k; x += E_THREADS) {
      int i = (int)(x / k), j = (int)(x - (long)i * k);
      out[x] = Vs[(long)i * np + s_perm[j]];
    }
  } else if (e.out_mode == 1) {
    for (long x = tid; x < (long)n * k; x += E_THREADS) {
      int j = (int)(x / n), i = (int)(x - (long)j * n);
      out[x] = cconj(Vs[(long)i * np + s_perm[j]]);
    }
  }
}

}  // namespace

template <typename R>
size_t eig_smem_bytes(int n_max) {
  int np = n_max + (n_max & 1);
  return 2 * (size_t)np * np * sizeof(cx<R>);
}
template size_t eig_smem_bytes<double>(int);
template size_t eig_smem_bytes<float>(int);

constexpr size_t EIG_SMEM_LIMIT = 200 * 1024;

template <typename R>
cudaError_t launch_eig(const EigDesc& e, const int* d_dims, cudaStream_t s, void* work, double* prof) {
  size_t bytes = eig_smem_bytes<R>(e.n_max);
  int use_smem = bytes <= EIG_SMEM_LIMIT;
  k_eig<R><<<1, E_THREADS, use_smem ? bytes : 0, s>>>(e, (int*)d_dims, (cx<R>*)work, use_smem, prof);
  return cudaGetLastError();
}
template cudaError_t launch_eig<double>(const EigDesc&, const int*, cudaStream_t, void*, double*);
template cudaError_t launch_eig<float>(const EigDesc&, const int*, cudaStream_t, void*, double*);

void init_kernel_attributes() {
  cudaFuncSetAttribute(k_eig<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_LIMIT);
  cudaFuncSetAttribute(k_eig<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_LIMIT);
}

}  // namespace qlb
