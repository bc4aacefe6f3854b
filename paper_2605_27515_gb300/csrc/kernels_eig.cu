// One-CTA cyclic Jacobi eigen-solve of a Hermitian (Gram) matrix that ends with
// the truncation decision of the bond it serves.
//
// Parallel (round-robin) ordering: in each of the np-1 rounds of a sweep the np
// indices form np/2 disjoint pairs, all rotated at once.  The rotation of pair
// (p, q) is J = [[c, sp], [-conj(sp), c]] with sp = s e^{i phi}, phi = arg G[p,q]
// and (c, s) the real symmetric Schur pair of [[G_pp, |G_pq|], [|G_pq|, G_qq]]
// (Golub & Van Loan, sym.schur2); G <- J^dag G J, V <- V J.  A pair is skipped
// when |G_pq| <= n eps sqrt(|G_pp G_qq|) (the relative criterion that keeps small
// eigenvalues of a Gram matrix accurate) or below an absolute floor of
// eps Tr G / 10, under the rounding already carried by the Gram matrix itself;
// a sweep with no rotation ends the solve.  At the sweep limit the solve is
// accepted when the off-diagonal norm left is below n eps Tr G.
//
// Each round has three barriers: rotation parameters, row update (J^dag G), and
// column update (G J, V J) which also writes the annihilated entries as exact
// zeros.  G and V sit in shared memory when 2 n^2 complex numbers of the runtime
// size fit, else in a global workspace.
//
// Instantiated for R = double (the FP64 form) and R = df64, a pair of floats
// (the mixed form): the same rotations on the FP32 pipes with ~48-bit significands.
// Input G and the output vectors are FP64 in both cases.

#include <type_traits>

#include "df64.cuh"
#include "qlb_internal.cuh"

namespace qlb {

namespace {

template <typename R>
struct Eps;
template <>
struct Eps<double> {
  static constexpr double v = 2.220446049250313e-16;
};
template <>
struct Eps<df64> {
  static constexpr double v = 1.4210854715202004e-14;  // 2^-46: double-float keeps ~46-48 bits
};

template <typename R>
__device__ __forceinline__ R to_r(double x) {
  return R(x);
}
template <typename R>
__device__ __forceinline__ double to_d(R x) {
  return (double)x;
}

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

template <typename R, int NT>
__global__ void __launch_bounds__(NT) k_eig(EigDesc e, int* __restrict__ d, cx<R>* work, int dyn_bytes,
                                           double* prof) {
  extern __shared__ unsigned char smem_raw[];
  const int n = dev_eval(e.n, d);
  const int tid = threadIdx.x;
  if (n <= 0) {
    if (tid == 0) d[e.dim_out] = 0;
    return;
  }
  const int np = n + (n & 1);
  const bool use_smem = 2L * np * np * (long)sizeof(cx<R>) <= (long)dyn_bytes;
  cx<R>* Gs = use_smem ? (cx<R>*)smem_raw : work;
  cx<R>* Vs = Gs + (long)np * np;
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

  const zd* G = (const zd*)e.G;
  for (long x = tid; x < (long)np * np; x += NT) {
    int i = (int)(x / np), j = (int)(x - (long)i * np);
    zd v = mk<double>(0, 0);
    if (i < n && j < n) v = G[(long)i * n + j];
    if (i == j) v.im = 0;
    Gs[x] = mk<R>(to_r<R>(v.re), to_r<R>(v.im));
    Vs[x] = mk<R>(to_r<R>(i == j ? 1.0 : 0.0), to_r<R>(0.0));
  }
  if (tid == 0) {
    s_bad = 0;
    double tr = 0;
    for (int i = 0; i < n; i++) tr += fabs(G[(long)i * n + i].re);
    // absolute floor eps Tr G / 10: G = M M^dag formed in floating point already
    // carries errors of order eps Tr G in every entry, so couplings below a tenth
    // of that move no eigenvalue or vector beyond what G itself fixes, and
    // rotating them only chases rounding noise (among the null directions of a
    // rank-deficient G above all).  Should noise still keep rotating, the solve
    // stops at the sweep limit and is accepted when the off-diagonal norm left is
    // below n eps Tr G.
    s_thr = to_r<R>(0.1 * Eps<R>::v * tr);
    s_tr = tr;
  }
  __syncthreads();
  const R abs_thr = s_thr;
  // relative floor: rounding in the row/column updates leaves off-diagonals of
  // order n eps sqrt(G_pp G_qq); asking for less would rotate noise forever
  const R rel_tol = to_r<R>(Eps<R>::v * (double)(n > 8 ? n : 8));
  const R zero = to_r<R>(0.0), one = to_r<R>(1.0);

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
        R c = one, s = zero;
        cx<R> sp = mk<R>(zero, zero);
        bool rot = false;
        if (q < n) {
          R a = Gs[(long)p * np + p].re, b = Gs[(long)q * np + q].re;
          cx<R> gpq = Gs[(long)p * np + q];
          R x = sqrt(cabs2(gpq));
          if (x > rel_tol * sqrt(fabs(a * b)) && x > abs_thr && x > zero) {
            R tau = (b - a) / (x + x);
            R t = fabs(tau) > to_r<R>(1e15) ? to_r<R>(0.5) / tau
                                            : (tau >= zero ? one : -one) / (fabs(tau) + sqrt(one + tau * tau));
            c = one / sqrt(one + t * t);
            s = t * c;
            R sx = s / x;
            sp = mk<R>(sx * gpq.re, sx * gpq.im);
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
      for (int w = tid; w < npairs * np; w += NT) {
        int t = w / np, j = w - t * np;
        int p = rp[t];
        if (p < 0) continue;
        int q = rq[t];
        R c = rc[t];
        cx<R> sp = rsp[t];
        cx<R> gp = Gs[(long)p * np + j], gq = Gs[(long)q * np + j];
        Gs[(long)p * np + j] = csub(cscale(gp, c), cmul(sp, gq));
        Gs[(long)q * np + j] = cadd(cmul(cconj(sp), gp), cscale(gq, c));
      }
      __syncthreads();
      // columns: G <- G J, V <- V J; the pair's off-diagonal becomes an exact zero
      for (int w = tid; w < npairs * np; w += NT) {
        int t = w / np, i = w - t * np;
        int p = rp[t];
        if (p < 0) continue;
        int q = rq[t];
        R c = rc[t];
        cx<R> sp = rsp[t];
        cx<R> gp = Gs[(long)i * np + p], gq = Gs[(long)i * np + q];
        cx<R> np_ = csub(cscale(gp, c), cmul(cconj(sp), gq));
        cx<R> nq_ = cadd(cmul(sp, gp), cscale(gq, c));
        if (i == p) {
          np_.im = zero;
          nq_ = mk<R>(zero, zero);
        } else if (i == q) {
          np_ = mk<R>(zero, zero);
          nq_.im = zero;
        }
        Gs[(long)i * np + p] = np_;
        Gs[(long)i * np + q] = nq_;
        cx<R> vp = Vs[(long)i * np + p], vq = Vs[(long)i * np + q];
        Vs[(long)i * np + p] = csub(cscale(vp, c), cmul(cconj(sp), vq));
        Vs[(long)i * np + q] = cadd(cmul(sp, vp), cscale(vq, c));
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
    for (long x = tid; x < (long)n * n; x += NT) {
      int i = (int)(x / n), j = (int)(x - (long)i * n);
      if (i != j) acc += to_d(cabs2(Gs[(long)i * np + j]));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) atomicAdd(&s_off, acc);
    __syncthreads();
    double lim = (double)n * Eps<R>::v * s_tr;
    unconverged = !(sqrt(s_off) <= lim);
  }
  if (prof && tid == 0) {
    atomicAdd(prof, 40.0 * (double)np * (double)total_rot);
    atomicAdd(prof + QLB_K_COUNT, 2.0 * sizeof(zd) * (double)n * (double)n);
  }

  // eigenvalues, sorted descending (stable on index)
  for (int i = tid; i < n; i += NT) {
    double li = to_d(Gs[(long)i * np + i].re);
    if (!isfinite(li)) s_bad = 1;
    int rank = 0;
    for (int j = 0; j < n; j++) {
      double lj = to_d(Gs[(long)j * np + j].re);
      if (lj > li || (lj == li && j < i)) rank++;
    }
    s_perm[rank] = i;
  }
  __syncthreads();
  for (int r = tid; r < n; r += NT) {
    double l = to_d(Gs[(long)s_perm[r] * np + s_perm[r]].re);
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
  zd* out = (zd*)e.out;
  if (e.out_mode == 0) {
    for (long x = tid; x < (long)n * k; x += NT) {
      int i = (int)(x / k), j = (int)(x - (long)i * k);
      cx<R> v = Vs[(long)i * np + s_perm[j]];
      out[x] = mk<double>(to_d(v.re), to_d(v.im));
    }
  } else if (e.out_mode == 1) {
    for (long x = tid; x < (long)n * k; x += NT) {
      int j = (int)(x / n), i = (int)(x - (long)j * n);
      cx<R> v = Vs[(long)i * np + s_perm[j]];
      out[x] = mk<double>(to_d(v.re), -to_d(v.im));
    }
  }
}

constexpr size_t EIG_SMEM_LIMIT = 200 * 1024;

template <typename R, int NT>
void set_attr() {
  cudaFuncSetAttribute(k_eig<R, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_LIMIT);
}

}  // namespace

template <typename R>
size_t eig_smem_bytes(int n_max) {
  int np = n_max + (n_max & 1);
  return 2 * (size_t)np * np * sizeof(cx<R>);
}
template size_t eig_smem_bytes<double>(int);
template size_t eig_smem_bytes<df64>(int);

template <typename R>
cudaError_t launch_eig(const EigDesc& e, const int* d_dims, cudaStream_t s, void* work, double* prof) {
  size_t want = eig_smem_bytes<R>(e.n_max);
  int dyn = (int)(want <= EIG_SMEM_LIMIT ? want : EIG_SMEM_LIMIT);
  // FP64: the DFMA pipe bounds the rotations, a few warps keep it busy.  Double-
  // float: long dependent FP32 chains per rotation, so a full CTA of warps hides
  // their latency.
  constexpr bool wide = std::is_same<R, df64>::value;
  if (e.n_max <= 24)
    k_eig<R, 128><<<1, 128, dyn, s>>>(e, (int*)d_dims, (cx<R>*)work, dyn, prof);
  else if (wide)
    k_eig<R, 1024><<<1, 1024, dyn, s>>>(e, (int*)d_dims, (cx<R>*)work, dyn, prof);
  else if (e.n_max <= 64)
    k_eig<R, 256><<<1, 256, dyn, s>>>(e, (int*)d_dims, (cx<R>*)work, dyn, prof);
  else
    k_eig<R, 512><<<1, 512, dyn, s>>>(e, (int*)d_dims, (cx<R>*)work, dyn, prof);
  return cudaGetLastError();
}
template cudaError_t launch_eig<double>(const EigDesc&, const int*, cudaStream_t, void*, double*);
template cudaError_t launch_eig<df64>(const EigDesc&, const int*, cudaStream_t, void*, double*);

void init_kernel_attributes() {
  set_attr<double, 128>();
  set_attr<double, 256>();
  set_attr<double, 512>();
  set_attr<df64, 128>();
  set_attr<df64, 256>();
  set_attr<df64, 512>();
  set_attr<df64, 1024>();
}

}  // namespace qlb
