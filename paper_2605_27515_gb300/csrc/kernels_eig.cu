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
// eps Tr G / 10, under the rounding already carried by the Gram matrix itself.
// (A looser floor for pairs of tiny diagonals was tried and dropped: directions of
// relative weight ~1e-15 are real content that the untruncated form must keep to
// reach 1e-10 in the observables.)  A sweep with no rotation ends the solve.  At
// the sweep limit the solve is accepted when the off-diagonal norm left is below
// n eps Tr G.
//
// Each round has three barriers: rotation parameters, row update (J^dag G), and
// column update (G J, V J) which also writes the annihilated entries as exact
// zeros.  G and V sit in shared memory when 2 n^2 complex numbers of the runtime
// size fit, else in a global workspace.
//
// Instantiated for R = double (the FP64 form) and R = df64, a pair of floats
// (the mixed form): the same rotations on the FP32 pipes with ~48-bit significands.
// Input G and the output vectors are FP64 in both cases.

#include <cooperative_groups.h>

#include <type_traits>

#include "df64.cuh"
#include "qlb_internal.cuh"

namespace qlb {

namespace {

// The updates of a rotation, c x - s y and s x + c y (real c, complex s), written
// as fused multiply-adds: FMAs in FP64, multiply-adds with one renormalisation in
// double-float (about 40 % fewer FP32 instructions than separate products and
// sums, at the same ~2^-44 relative accuracy).
__device__ __forceinline__ double rmac(double c, double a, double b) { return fma(a, b, c); }
__device__ __forceinline__ df64 rmac(df64 c, df64 a, df64 b) { return df_mac(c, a, b); }
template <typename R>
__device__ __forceinline__ cx<R> rot_cx_minus_sy(cx<R> x, R c, cx<R> s, cx<R> y) {
  return mk<R>(rmac(rmac(c * x.re, -s.re, y.re), s.im, y.im), rmac(rmac(c * x.im, -s.re, y.im), -s.im, y.re));
}
template <typename R>
__device__ __forceinline__ cx<R> rot_sx_plus_cy(cx<R> s, cx<R> x, R c, cx<R> y) {
  return mk<R>(rmac(rmac(c * y.re, s.re, x.re), -s.im, x.im), rmac(rmac(c * y.im, s.re, x.im), s.im, x.re));
}

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

// Shared end of both eigen-solvers: eigenvalues lam[0..n) (unsorted, in shared
// memory) and eigenvectors V(i, j) = V[i * vr + j * vc] (component i of vector j)
// become the sorted weights, the kept count k (written to dims), the weight
// statistics and the kept vectors in the requested layout.
template <typename R, int NT>
__device__ void eig_finish(const EigDesc& e, int* d, int n, const double* lam, const cx<R>* V, long vr, long vc,
                           bool unconverged, int* s_perm, double* s_w, int* s_k, int* s_bad) {
  const int tid = threadIdx.x;
  // eigenvalues, sorted descending (stable on index)
  for (int i = tid; i < n; i += NT) {
    double li = lam[i];
    if (!isfinite(li)) *s_bad = 1;
    int rank = 0;
    for (int j = 0; j < n; j++) {
      double lj = lam[j];
      if (lj > li || (lj == li && j < i)) rank++;
    }
    s_perm[rank] = i;
  }
  __syncthreads();
  for (int r = tid; r < n; r += NT) {
    double l = lam[s_perm[r]];
    s_w[r] = l > 0.0 ? l : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    int cap = dev_eval(e.cap, d);
    if (cap < 1) cap = 1;
    int k = *s_bad ? 1 : keep_count_dev(s_w, n, e.tol, cap, e.gap);
    *s_k = k;
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
    if (e.solver_stats) {
      atomicAdd(e.solver_stats + 0, 1.0);
      atomicAdd(e.solver_stats + 2, (double)n);
      atomicAdd(e.solver_stats + 3, (double)k);
      // largest runtime size: non-negative doubles order like their bit patterns
      atomicMax((unsigned long long*)(e.solver_stats + 6), (unsigned long long)__double_as_longlong((double)n));
    }
    if (e.err) {
      if (unconverged) atomicOr(e.err, 1);
      if (*s_bad || !isfinite(total)) atomicOr(e.err, 2);
    }
  }
  __syncthreads();
  const int k = *s_k;
  zd* out = (zd*)e.out;
  if (e.out_mode == 0) {
    for (long x = tid; x < (long)n * k; x += NT) {
      int i = (int)(x / k), j = (int)(x - (long)i * k);
      cx<R> v = V[i * vr + s_perm[j] * vc];
      out[x] = mk<double>(to_d(v.re), to_d(v.im));
    }
  } else if (e.out_mode == 1) {
    for (long x = tid; x < (long)n * k; x += NT) {
      int j = (int)(x / n), i = (int)(x - (long)j * n);
      cx<R> v = V[i * vr + s_perm[j] * vc];
      out[x] = mk<double>(to_d(v.re), -to_d(v.im));
    }
  }
}

template <typename R, int NT, bool GRP = false>
__global__ void __launch_bounds__(NT) k_eig(EigDesc e, int* __restrict__ d, cx<R>* work, int dyn_bytes,
                                           double* prof, const EigDesc* __restrict__ grp) {
  extern __shared__ unsigned char smem_raw[];
  if constexpr (GRP) {  // grouped launch: one CTA per member (blockIdx.y)
    e = grp[blockIdx.y];
    d = e.dims;
    work = (cx<R>*)e.work;
  }
  if (e.gate && *e.gate == 0) return;  // the zip-up range basis already served this bond
  const int n = dev_eval(e.n, d);
  const int tid = threadIdx.x;
  if (n <= 0) {
    if (tid == 0) d[e.dim_out] = 0;
    return;
  }
  const int np = n + (n & 1);
  const bool use_smem = 2L * np * np * (long)sizeof(cx<R>) <= (long)dyn_bytes;
  if (!use_smem && e.solver_stats && tid == 0) atomicAdd(e.solver_stats + 5, 1.0);
  cx<R>* Gs = use_smem ? (cx<R>*)smem_raw : work;
  cx<R>* Vs = Gs + (long)np * np;
  __shared__ R rc[256];
  __shared__ cx<R> rsp[256];
  __shared__ int rp[256], rq[256];
  __shared__ int n_rot;
  __shared__ int s_perm[512];
  __shared__ double s_w[512];
  __shared__ double s_lam[512];
  __shared__ int s_k;
  __shared__ int s_bad;
  __shared__ R s_thr;
  __shared__ double s_tr;
  __shared__ double s_off;
  __shared__ int s_any;

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
        Gs[(long)p * np + j] = rot_cx_minus_sy(gp, c, sp, gq);
        Gs[(long)q * np + j] = rot_sx_plus_cy(cconj(sp), gp, c, gq);
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
        cx<R> np_ = rot_cx_minus_sy(gp, c, cconj(sp), gq);
        cx<R> nq_ = rot_sx_plus_cy(sp, gp, c, gq);
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
        Vs[(long)i * np + p] = rot_cx_minus_sy(vp, c, cconj(sp), vq);
        Vs[(long)i * np + q] = rot_sx_plus_cy(sp, vp, c, vq);
      }
      __syncthreads();
    }
    int nr = n_rot;
    total_rot += nr;
    __syncthreads();
    if (nr == 0) break;
    // A sweep that rotates nothing leaves G as it is, so it rotates nothing exactly
    // when no pair passes the rotation test on the current G: test every pair at
    // once (the same expressions) instead of spending a sweep of rounds on it.
    if (tid == 0) s_any = 0;
    __syncthreads();
    for (long w = tid; w < (long)n * n; w += NT) {
      const int p = (int)(w / n), q = (int)(w - (long)p * n);
      if (q <= p) continue;
      R a = Gs[(long)p * np + p].re, b = Gs[(long)q * np + q].re;
      R x = sqrt(cabs2(Gs[(long)p * np + q]));
      if (x > rel_tol * sqrt(fabs(a * b)) && x > abs_thr && x > zero) s_any = 1;
    }
    __syncthreads();
    if (!s_any) break;
  }
  bool unconverged = false;
  const bool at_limit = sweep >= e.max_sweeps;
  if (e.solver_stats && tid == 0) {
    atomicAdd(e.solver_stats + 1, (double)(at_limit ? e.max_sweeps : sweep + 1));
    if (at_limit) atomicAdd(e.solver_stats + 4, 1.0);
  }
  if (at_limit) {
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

  for (int i = tid; i < n; i += NT) s_lam[i] = to_d(Gs[(long)i * np + i].re);
  __syncthreads();
  eig_finish<R, NT>(e, d, n, s_lam, Vs, np, 1, unconverged, s_perm, s_w, &s_k, &s_bad);
}

// The same cyclic Jacobi solve spread over a thread-block cluster of C CTAs (C SMs).
// On this GPU one SM retires two FP64 FMAs per clock, and the one-CTA solve above
// saturates that pipe, so the solve is split by rows: CTA r holds rows
// [r * rpb, (r + 1) * rpb) of G and of V in its shared memory, and the cluster
// runs the identical rotation schedule, thresholds and truncation rule.  Each
// round takes two cluster barriers:
//   A  the owner of row p computes the rotation of pair (p, q) (G_qq read from
//      q's owner through distributed shared memory) and writes it into the
//      rotation table of every CTA;
//      -- cluster barrier --
//   B  rows (J^dag G): each CTA writes its rows of the next buffer, reading the
//      partner row from its owner (the current buffer is not written in a round);
//   C  columns (G J, V J) on its own rows of the next buffer, with the annihilated
//      entries written as exact zeros;
//      -- cluster barrier --
// The eigenvalues are then gathered by every CTA, which all take the same
// truncation decision; each CTA writes the kept vectors of its own rows.
template <typename R>
struct JRot {
  R c;
  cx<R> sp;
  int p, q;  // p < 0: the pair is not rotated this round
};

constexpr int EIG_CL_MAX_NP = 256;

template <typename R, int NT, int C, bool GRP = false>
__global__ void __launch_bounds__(NT) k_eig_cl(EigDesc e, int* __restrict__ d, double* prof,
                                              const EigDesc* __restrict__ grp) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ unsigned char smem_raw[];
  if constexpr (GRP) {  // grouped launch: one cluster per member (blockIdx.y; the cluster spans x)
    e = grp[blockIdx.y];
    d = e.dims;
  }
  if (e.gate && *e.gate == 0) return;  // the zip-up range basis already served this bond
  const int n = dev_eval(e.n, d);
  const int tid = threadIdx.x;
  const int rank = (int)cluster.block_rank();
  if (n <= 0) {
    if (rank == 0 && tid == 0) d[e.dim_out] = 0;
    return;
  }
  const int np = n + (n & 1);
  const int rpb = (np + C - 1) / C;
  const int r0 = rank * rpb;
  const int r1 = min(np, r0 + rpb);
  const int nloc = max(0, r1 - r0);
  cx<R>* Gb0 = (cx<R>*)smem_raw;
  cx<R>* Gb1 = Gb0 + (long)rpb * np;
  cx<R>* Vl = Gb1 + (long)rpb * np;
  __shared__ JRot<R> rot[EIG_CL_MAX_NP / 2];
  __shared__ int cnt[2], chk[2];
  __shared__ double s_part;
  __shared__ double s_lam[EIG_CL_MAX_NP];
  __shared__ int s_perm[EIG_CL_MAX_NP];
  __shared__ double s_w[EIG_CL_MAX_NP];
  __shared__ int s_k, s_bad;
  __shared__ R s_thr;
  __shared__ double s_tr;
  const R zero = to_r<R>(0.0), one = to_r<R>(1.0);

  const zd* G = (const zd*)e.G;
  for (long x = tid; x < (long)nloc * np; x += NT) {
    int li = (int)(x / np), j = (int)(x - (long)li * np);
    int i = r0 + li;
    zd v = mk<double>(0, 0);
    if (i < n && j < n) v = G[(long)i * n + j];
    if (i == j) v.im = 0;
    Gb0[x] = mk<R>(to_r<R>(v.re), to_r<R>(v.im));
    Vl[x] = mk<R>(to_r<R>(i == j ? 1.0 : 0.0), zero);
  }
  if (tid == 0) {
    s_bad = 0;
    cnt[0] = cnt[1] = 0;
    double tr = 0;
    for (int i = 0; i < n; i++) tr += fabs(G[(long)i * n + i].re);
    s_thr = to_r<R>(0.1 * Eps<R>::v * tr);  // the same floors as the one-CTA solve
    s_tr = tr;
  }
  cluster.sync();
  const R abs_thr = s_thr;
  const R rel_tol = to_r<R>(Eps<R>::v * (double)(n > 8 ? n : 8));
  const int npairs = np / 2;
  int cur = 0;
  int sweep = 0;
  long total_rot = 0;
  for (; sweep < e.max_sweeps; sweep++) {
    const int par = sweep & 1;
    if (tid == 0) cnt[par] = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; round++) {
      cx<R>* Gc = cur ? Gb1 : Gb0;
      cx<R>* Gn = cur ? Gb0 : Gb1;
      // A: rotations of the pairs whose p row is ours, published cluster-wide
      for (int t = tid; t < npairs; t += NT) {
        int p = rr_player(t, round, np), q = rr_player(np - 1 - t, round, np);
        if (p > q) {
          int tmp = p;
          p = q;
          q = tmp;
        }
        if (p < r0 || p >= r1) continue;
        R c = one;
        cx<R> sp = mk<R>(zero, zero);
        bool rotf = false;
        if (q < n) {
          R a = Gc[(long)(p - r0) * np + p].re;
          cx<R> gpq = Gc[(long)(p - r0) * np + q];
          const int oq = q / rpb;
          const cx<R>* Gq = cluster.map_shared_rank(Gc, oq);
          R b = Gq[(long)(q - oq * rpb) * np + q].re;
          R x = sqrt(cabs2(gpq));
          if (x > rel_tol * sqrt(fabs(a * b)) && x > abs_thr && x > zero) {
            R tau = (b - a) / (x + x);
            R tt = fabs(tau) > to_r<R>(1e15) ? to_r<R>(0.5) / tau
                                              : (tau >= zero ? one : -one) / (fabs(tau) + sqrt(one + tau * tau));
            c = one / sqrt(one + tt * tt);
            R sx = (tt * c) / x;
            sp = mk<R>(sx * gpq.re, sx * gpq.im);
            rotf = true;
          }
        }
        JRot<R> rr;
        rr.c = c;
        rr.sp = sp;
        rr.p = rotf ? p : -1;
        rr.q = q;
        for (int k = 0; k < C; k++) cluster.map_shared_rank(rot, k)[t] = rr;
        if (rotf) atomicAdd(&cnt[par], 1);
      }
      cluster.sync();
      // B: rows of J^dag G into the next buffer
      for (long w = tid; w < (long)nloc * np; w += NT) {
        const int li = (int)(w / np), j = (int)(w - (long)li * np);
        const int i = r0 + li;
        const int pos = i == 0 ? 0 : 1 + ((i - 1 - round) % (np - 1) + (np - 1)) % (np - 1);
        const JRot<R> rr = rot[pos < npairs ? pos : np - 1 - pos];
        cx<R> gi = Gc[w];
        cx<R> out = gi;
        if (rr.p >= 0) {
          const int partner = i == rr.p ? rr.q : rr.p;
          const int op = partner / rpb;
          const cx<R> gx = cluster.map_shared_rank(Gc, op)[(long)(partner - op * rpb) * np + j];
          out = i == rr.p ? rot_cx_minus_sy(gi, rr.c, rr.sp, gx) : rot_sx_plus_cy(cconj(rr.sp), gx, rr.c, gi);
        }
        Gn[w] = out;
      }
      __syncthreads();
      // C: columns G J, V J on our rows; the pair's off-diagonal becomes an exact zero
      for (long w = tid; w < (long)nloc * npairs; w += NT) {
        const int li = (int)(w / npairs), t = (int)(w - (long)li * npairs);
        const JRot<R> rr = rot[t];
        if (rr.p < 0) continue;
        const int p = rr.p, q = rr.q, i = r0 + li;
        cx<R> gp = Gn[(long)li * np + p], gq = Gn[(long)li * np + q];
        cx<R> np_ = rot_cx_minus_sy(gp, rr.c, cconj(rr.sp), gq);
        cx<R> nq_ = rot_sx_plus_cy(rr.sp, gp, rr.c, gq);
        if (i == p) {
          np_.im = zero;
          nq_ = mk<R>(zero, zero);
        } else if (i == q) {
          np_ = mk<R>(zero, zero);
          nq_.im = zero;
        }
        Gn[(long)li * np + p] = np_;
        Gn[(long)li * np + q] = nq_;
        cx<R> vp = Vl[(long)li * np + p], vq = Vl[(long)li * np + q];
        Vl[(long)li * np + p] = rot_cx_minus_sy(vp, rr.c, cconj(rr.sp), vq);
        Vl[(long)li * np + q] = rot_sx_plus_cy(rr.sp, vp, rr.c, vq);
      }
      cluster.sync();
      cur ^= 1;
    }
    int nr = 0;
    for (int k = 0; k < C; k++) nr += *cluster.map_shared_rank(&cnt[par], k);
    total_rot += nr;
    if (nr == 0) break;
    // as in the one-CTA solve: a sweep would rotate nothing exactly when no pair
    // passes the test on the current G; each CTA tests the pairs of its rows
    {
      const cx<R>* Gc = cur ? Gb1 : Gb0;
      if (tid == 0) chk[par] = 0;
      __syncthreads();
      for (long w = tid; w < (long)nloc * np; w += NT) {
        const int li = (int)(w / np), q = (int)(w - (long)li * np);
        const int p = r0 + li;
        if (p >= n || q >= n || q <= p) continue;
        const int oq = q / rpb;
        R a = Gc[(long)li * np + p].re;
        R b = cluster.map_shared_rank(Gc, oq)[(long)(q - oq * rpb) * np + q].re;
        R x = sqrt(cabs2(Gc[(long)li * np + q]));
        if (x > rel_tol * sqrt(fabs(a * b)) && x > abs_thr && x > zero) chk[par] = 1;
      }
      cluster.sync();
      int any = 0;
      for (int k = 0; k < C; k++) any += *cluster.map_shared_rank(&chk[par], k);
      if (!any) break;
    }
  }
  cx<R>* Gc = cur ? Gb1 : Gb0;
  bool unconverged = false;
  const bool at_limit = sweep >= e.max_sweeps;
  if (at_limit) {
    // accept a solve whose remaining couplings are at the rounding level
    if (tid == 0) s_part = 0.0;
    __syncthreads();
    double acc = 0.0;
    for (long x = tid; x < (long)nloc * np; x += NT) {
      int li = (int)(x / np), j = (int)(x - (long)li * np);
      int i = r0 + li;
      if (i < n && j < n && i != j) acc += to_d(cabs2(Gc[x]));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) atomicAdd(&s_part, acc);
    cluster.sync();
    double off = 0.0;
    for (int k = 0; k < C; k++) off += *cluster.map_shared_rank(&s_part, k);
    unconverged = !(sqrt(off) <= (double)n * Eps<R>::v * s_tr);
  }
  // every CTA gathers the eigenvalues and takes the same truncation decision
  for (int i = tid; i < n; i += NT) {
    const int oi = i / rpb;
    s_lam[i] = to_d(cluster.map_shared_rank(Gc, oi)[(long)(i - oi * rpb) * np + i].re);
  }
  cluster.sync();  // no CTA leaves while another still reads its shared memory
  for (int i = tid; i < n; i += NT) {
    double li = s_lam[i];
    if (!isfinite(li)) s_bad = 1;
    int rk = 0;
    for (int j = 0; j < n; j++) {
      double lj = s_lam[j];
      if (lj > li || (lj == li && j < i)) rk++;
    }
    s_perm[rk] = i;
  }
  __syncthreads();
  for (int r = tid; r < n; r += NT) {
    double l = s_lam[s_perm[r]];
    s_w[r] = l > 0.0 ? l : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    int cap = dev_eval(e.cap, d);
    if (cap < 1) cap = 1;
    int k = s_bad ? 1 : keep_count_dev(s_w, n, e.tol, cap, e.gap);
    s_k = k;
    if (rank == 0) {
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
      if (e.solver_stats) {
        atomicAdd(e.solver_stats + 0, 1.0);
        atomicAdd(e.solver_stats + 1, (double)(at_limit ? e.max_sweeps : sweep + 1));
        atomicAdd(e.solver_stats + 2, (double)n);
        atomicAdd(e.solver_stats + 3, (double)k);
        if (at_limit) atomicAdd(e.solver_stats + 4, 1.0);
        atomicAdd(e.solver_stats + 5, 1.0);  // a multi-SM solve
        atomicMax((unsigned long long*)(e.solver_stats + 6), (unsigned long long)__double_as_longlong((double)n));
      }
      if (prof) {
        atomicAdd(prof, 40.0 * (double)np * (double)total_rot);
        atomicAdd(prof + QLB_K_COUNT, 2.0 * sizeof(zd) * (double)n * (double)n);
      }
    }
  }
  __syncthreads();
  const int k = s_k;
  zd* out = (zd*)e.out;
  const int rl = max(0, min(r1, n) - r0);
  if (e.out_mode == 0) {
    for (long x = tid; x < (long)rl * k; x += NT) {
      int li = (int)(x / k), j = (int)(x - (long)li * k);
      cx<R> v = Vl[(long)li * np + s_perm[j]];
      out[(long)(r0 + li) * k + j] = mk<double>(to_d(v.re), to_d(v.im));
    }
  } else if (e.out_mode == 1) {
    for (long x = tid; x < (long)rl * k; x += NT) {
      int li = (int)(x / k), j = (int)(x - (long)li * k);
      cx<R> v = Vl[(long)li * np + s_perm[j]];
      out[(long)j * n + (r0 + li)] = mk<double>(to_d(v.re), -to_d(v.im));
    }
  }
}

// One-CTA Hermitian eigen-solve by Householder tridiagonalisation and implicit QL
// (the FP64 form at sizes whose matrices fit in shared memory).  Cyclic Jacobi
// spends ~30 n^3 flops and 3 barriers per round over ~10 sweeps of n - 1 rounds;
// this solver ~15 n^3 flops, 3 barriers per column and one per QL step, but the
// QL bulge chase is a serial chain of ~n^2 dependent rotations, so it is used
// only for small planned sizes (measured on GB300: 20-200 us per solve at
// n <= 64; at n ~ 128, with its matrices in global memory, the chain made it
// slower than Jacobi).
//
// 1. Tridiagonalisation (Golub & Van Loan, Alg. 8.3.1, complex form).  For column
//    k the reflector H = I - tau v v^dag with v = x + e^{i phi} |x| e_1,
//    e^{i phi} = x_1 / |x_1|, tau = 1 / (|x| (|x| + |x_1|)) maps x = A[k+1:, k] to
//    -e^{i phi} |x| e_1.  The trailing block takes A <- H A H as
//    A - v w^dag - w v^dag with p = tau A v, w = p - (tau/2)(v^dag p) v, and
//    Q <- Q H accumulates Q (G = Q T Q^dag).
// 2. A diagonal phase matrix D turns the complex subdiagonal beta_k into |beta_k|:
//    d_0 = 1, d_{k+1} = d_k beta_k / |beta_k|; T' = D^dag T D is real symmetric.
// 3. Implicit QL with the Wilkinson-type shift from the leading 2x2 of the
//    unreduced block (Bowdler, Martin, Reinsch & Wilkinson, "The QR and QL
//    algorithms for symmetric matrices", 1968), rotations applied to the columns
//    of W = Q D, which ends as the eigenvectors of G.  Off-diagonals deflate below
//    eps (|d_m| + |d_m+1|) or below eps Tr G / 1000.
//
// Lane 0 of warp 0 runs the scalar QL recurrence; the other warps apply the
// rotations of the previous QL step to the rows of W meanwhile (double-buffered
// rotation lists, one barrier per QL step).  Q and W are stored transposed
// (Wt[j][i] = W[i][j]) so that a thread per row i reads consecutive words.
constexpr int HEEV_MAX_IT = 60;

template <int NT>
__global__ void __launch_bounds__(NT) k_heev(EigDesc e, int* __restrict__ d, zd* work, int dyn_bytes, double* prof) {
  extern __shared__ unsigned char smem_raw[];
  if (e.gate && *e.gate == 0) return;  // the zip-up range basis already served this bond
  const int n = dev_eval(e.n, d);
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  if (n <= 0) {
    if (tid == 0) d[e.dim_out] = 0;
    return;
  }
  const int np = n + (n & 1);
  const bool use_smem = 2L * np * np * (long)sizeof(zd) <= (long)dyn_bytes;
  if (!use_smem && e.solver_stats && tid == 0) atomicAdd(e.solver_stats + 5, 1.0);
  zd* A = use_smem ? (zd*)smem_raw : work;
  zd* Qt = A + (long)np * np;
  __shared__ zd s_v[512], s_p[512], s_u[512];
  __shared__ double s_d[512], s_e[512];
  __shared__ double s_rc[2][512], s_rs[2][512];
  __shared__ int s_rm[2], s_rn[2];
  __shared__ int s_done[2], s_fail;
  // per-pass flags are double-buffered: a thread still reading the flag of pass t
  // after the barrier must not see pass t+1's value
  __shared__ double s_tau[2], s_tr;
  __shared__ int s_skip[2];
  __shared__ int s_perm[512];
  __shared__ double s_w[512];
  __shared__ int s_k, s_bad;
  __shared__ int s_pass_count;
  const double eps = 2.220446049250313e-16;

  const zd* G = (const zd*)e.G;
  for (long x = tid; x < (long)n * n; x += NT) {
    int i = (int)(x / n), j = (int)(x - (long)i * n);
    zd v = G[x];
    if (i == j) v.im = 0.0;
    A[(long)i * np + j] = v;
    Qt[(long)i * np + j] = mk<double>(i == j ? 1.0 : 0.0, 0.0);
  }
  if (tid == 0) {
    s_bad = 0;
    s_fail = 0;
    double tr = 0.0;
    for (int i = 0; i < n; i++) tr += fabs(G[(long)i * n + i].re);
    s_tr = tr;
  }
  __syncthreads();

  // 1. tridiagonalisation, column by column
  double flops = 0.0;
  for (int k = 0; k + 2 < n; k++) {
    const int m = n - k - 1;  // trailing size
    const zd* rowk = A + (long)k * np + (k + 1);  // A[k][k+1..] = conj(x)
    if (tid < 32) {
      double s2 = 0.0;
      for (int i = lane; i < m; i += 32) s2 += cabs2(rowk[i]);
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      zd x0 = cconj(rowk[0]);
      double a0 = sqrt(cabs2(x0));
      double sig = sqrt(s2);
      zd ph = a0 > 0.0 ? cscale(x0, 1.0 / a0) : mk<double>(1.0, 0.0);
      if (s2 > 0.0) {
        for (int i = lane; i < m; i += 32) s_v[i] = i == 0 ? cscale(ph, a0 + sig) : cconj(rowk[i]);
      }
      __syncwarp();  // every lane has read row k before lane 0 overwrites A[k][k+1]
      if (lane == 0) {
        s_skip[k & 1] = !(s2 > 0.0);
        s_tau[k & 1] = s2 > 0.0 ? 1.0 / (sig * (sig + a0)) : 0.0;
        if (s2 > 0.0) {
          zd beta = cscale(ph, -sig);
          A[(long)(k + 1) * np + k] = beta;
          A[(long)k * np + (k + 1)] = cconj(beta);
        }
      }
    }
    __syncthreads();
    if (s_skip[k & 1]) continue;
    const double tau = s_tau[k & 1];
    const long o = (long)(k + 1) * np + (k + 1);  // trailing block origin
    // p = tau A v (A Hermitian: row i of A is the conjugate of column i) and u = Q v
    for (int i = tid; i < m; i += NT) {
      zd acc = mk<double>(0.0, 0.0);
      for (int j = 0; j < m; j++) cfma(acc, cconj(A[o + (long)j * np + i]), s_v[j]);
      s_p[i] = cscale(acc, tau);
    }
    for (int i = tid; i < n; i += NT) {
      zd acc = mk<double>(0.0, 0.0);
      for (int j = 0; j < m; j++) cfma(acc, Qt[(long)(k + 1 + j) * np + i], s_v[j]);
      s_u[i] = acc;
    }
    __syncthreads();
    // K = (tau/2) v^dag p, computed by every warp
    double kk = 0.0;
    for (int i = lane; i < m; i += 32) {
      zd a = s_v[i], b = s_p[i];
      kk += a.re * b.re + a.im * b.im;
    }
    for (int q = 16; q > 0; q >>= 1) kk += __shfl_xor_sync(0xffffffffu, kk, q);
    const double K = 0.5 * tau * kk;
    // A_trailing -= v w^dag + w v^dag,  Q[:, k+1:] -= tau u v^dag
    for (long x = tid; x < (long)m * m; x += NT) {
      int i = (int)(x / m), j = (int)(x - (long)i * m);
      zd vi = s_v[i], vj = s_v[j];
      zd wi = csub(s_p[i], cscale(vi, K)), wj = csub(s_p[j], cscale(vj, K));
      zd a = A[o + (long)i * np + j];
      a = csub(a, cmul(vi, cconj(wj)));
      a = csub(a, cmul(wi, cconj(vj)));
      A[o + (long)i * np + j] = a;
    }
    for (long x = tid; x < (long)m * n; x += NT) {
      int j = (int)(x / n), i = (int)(x - (long)j * n);
      long a = (long)(k + 1 + j) * np + i;
      Qt[a] = csub(Qt[a], cscale(cmul(s_u[i], cconj(s_v[j])), tau));
    }
    flops += 24.0 * m * m + 16.0 * (double)n * m;
    __syncthreads();
  }

  // 2. real tridiagonal T' = D^dag T D and W = Q D (rows of Qt scaled)
  if (tid == 0) {
    zd ph = mk<double>(1.0, 0.0);
    for (int k = 0; k < n; k++) {
      s_d[k] = A[(long)k * np + k].re;
      s_u[k] = ph;
      if (k + 1 < n) {
        zd b = cconj(A[(long)k * np + (k + 1)]);  // subdiagonal, read from the row kept exact
        double ab = sqrt(cabs2(b));
        s_e[k] = ab;
        if (ab > 0.0) ph = cmul(ph, cscale(b, 1.0 / ab));
      } else {
        s_e[k] = 0.0;
      }
    }
    s_done[0] = s_done[1] = 0;
    s_rn[0] = s_rn[1] = 0;
  }
  __syncthreads();
  for (long x = tid; x < (long)n * n; x += NT) {
    int j = (int)(x / n), i = (int)(x - (long)j * n);
    long a = (long)j * np + i;
    Qt[a] = cmul(Qt[a], s_u[j]);
  }
  __syncthreads();

  // 3. implicit QL; lane 0 of warp 0 produces the rotations of one QL step per
  // pass, the other warps apply those of the previous pass to the rows of W.
  zd* Wt = Qt;
  const double floor_abs = 1e-3 * eps * s_tr;
  // QL iterations allowed per eigenvalue (usually 1-3 are needed); the context's
  // sweep limit caps it as well, so a forced limit of 1 is observable here too
  const int it_limit = e.max_sweeps < HEEV_MAX_IT ? (e.max_sweeps > 0 ? e.max_sweeps : 1) : HEEV_MAX_IT;
  int ql_l = 0, ql_it = 0;
  long n_rot = 0;
  for (int t = 0;; t++) {
    const int b = t & 1;
    if (tid == 0) {
      int cnt = 0, mtop = 0;
      while (ql_l < n) {
        int m = ql_l;
        while (m < n - 1) {
          double dd = fabs(s_d[m]) + fabs(s_d[m + 1]);
          double em = fabs(s_e[m]);
          if (em <= eps * dd || em <= floor_abs) break;
          m++;
        }
        if (m == ql_l) {
          ql_l++;
          ql_it = 0;
          continue;
        }
        if (++ql_it > it_limit) {
          s_fail = 1;
          s_e[m - 1] = 0.0;  // give up on this coupling; flagged as unconverged
          continue;
        }
        const int l = ql_l;
        double g = (s_d[l + 1] - s_d[l]) / (2.0 * s_e[l]);
        double r = hypot(g, 1.0);
        g = s_d[m] - s_d[l] + s_e[l] / (g + (g >= 0.0 ? r : -r));
        double sn = 1.0, cs = 1.0, p = 0.0;
        bool under = false;
        mtop = m;
        for (int i = m - 1; i >= l; i--) {
          double f = sn * s_e[i], bb = cs * s_e[i];
          r = hypot(f, g);
          s_e[i + 1] = r;
          if (r == 0.0) {
            s_d[i + 1] -= p;
            s_e[m] = 0.0;
            under = true;
            break;
          }
          sn = f / r;
          cs = g / r;
          g = s_d[i + 1] - p;
          r = (s_d[i] - g) * sn + 2.0 * cs * bb;
          p = sn * r;
          s_d[i + 1] = g + p;
          g = cs * r - bb;
          s_rc[b][cnt] = cs;
          s_rs[b][cnt] = sn;
          cnt++;
        }
        if (!under) {
          s_d[l] -= p;
          s_e[l] = g;
          s_e[m] = 0.0;
        }
        break;  // one QL step per pass
      }
      s_rm[b] = mtop;
      s_rn[b] = cnt;
      n_rot += cnt;
      s_done[b] = ql_l >= n;
    } else if (tid >= 32 && t > 0) {
      // rotations (i, i+1) for i = m-1, m-2, ... of the previous pass: keep the
      // running entry of column i+1 in registers
      const int pb = b ^ 1;
      const int cnt = s_rn[pb];
      if (cnt > 0) {
        const int m = s_rm[pb];
        for (int row = tid - 32; row < n; row += NT - 32) {
          zd cur = Wt[(long)m * np + row];
          for (int j = 0; j < cnt; j++) {
            const int i = m - 1 - j;
            const double cs = s_rc[pb][j], sn = s_rs[pb][j];
            zd a = Wt[(long)i * np + row];
            Wt[(long)(i + 1) * np + row] = mk<double>(sn * a.re + cs * cur.re, sn * a.im + cs * cur.im);
            cur = mk<double>(cs * a.re - sn * cur.re, cs * a.im - sn * cur.im);
          }
          Wt[(long)(m - cnt) * np + row] = cur;
        }
      }
    }
    __syncthreads();
    if (s_done[b]) {  // a finishing pass produces no rotations
      if (tid == 0) s_pass_count = t + 1;
      break;
    }
  }
  __syncthreads();
  if (e.solver_stats && tid == 0) {
    atomicAdd(e.solver_stats + 1, (double)(s_pass_count));
    if (s_fail) atomicAdd(e.solver_stats + 4, 1.0);
  }
  if (prof && tid == 0) {
    atomicAdd(prof, flops + 8.0 * (double)n * (double)n_rot);
    atomicAdd(prof + QLB_K_COUNT, 2.0 * sizeof(zd) * (double)n * (double)n);
  }
  eig_finish<double, NT>(e, d, n, s_d, Wt, 1, np, s_fail != 0, s_perm, s_w, &s_k, &s_bad);
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

// Dynamic shared memory of the QL solver: its static arrays take ~55 KB of the
// 227 KB a CTA may hold, so A and W stay in shared memory up to n ~ 70.
constexpr size_t HEEV_SMEM_LIMIT = 160 * 1024;
constexpr int HEEV_N_MAX = 64;

size_t eig_workspace_elems(int n_max) {
  if (n_max <= EIG_CL_MAX_NP) return 1;  // cluster solves keep everything in shared memory
  int np = n_max + (n_max & 1);
  size_t need = 2 * (size_t)np * np;
  size_t limit = n_max <= HEEV_N_MAX ? HEEV_SMEM_LIMIT : EIG_SMEM_LIMIT;
  return need * sizeof(zd) > limit ? need : 1;
}

// Workspace a member of planned size n_max needs when a grouped launch serves it
// with the kernel picked for the group's largest planned size group_n_max: the
// one-CTA kernel (group_n_max <= 24 or above the cluster range) sizes its shared
// memory for group_n_max, capped, and falls back to the member's workspace for
// problems that do not fit; the cluster kernels need none.
size_t eig_group_workspace_elems(int n_max, int group_n_max) {
  if (group_n_max > 24 && group_n_max <= EIG_CL_MAX_NP) return 1;
  const size_t dyn = std::min(eig_smem_bytes<double>(group_n_max), (size_t)EIG_SMEM_LIMIT);
  const int np = n_max + (n_max & 1);
  const size_t need = 2 * (size_t)np * np;
  return need * sizeof(zd) > dyn ? need : 1;
}

template <typename R, int C>
cudaError_t launch_eig_cl(const EigDesc& e, const int* d_dims, cudaStream_t s, double* prof,
                          const EigDesc* grp = nullptr, int S = 1) {
  const int np = e.n_max + (e.n_max & 1);
  const int rpb = (np + C - 1) / C;
  size_t dyn = 3 * (size_t)rpb * np * sizeof(cx<R>);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, S, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (grp) return cudaLaunchKernelEx(&cfg, k_eig_cl<R, 256, C, true>, e, (int*)d_dims, prof, grp);
  return cudaLaunchKernelEx(&cfg, k_eig_cl<R, 256, C, false>, e, (int*)d_dims, prof, grp);
}

template <typename R>
cudaError_t launch_eig(const EigDesc& e, const int* d_dims, cudaStream_t s, void* work, double* prof) {
  // Jacobi in both precisions.  The Householder + QL solve (k_heev) is not used by
  // the step: on the literal cat_r9 map its absolute-accuracy vectors seeded a
  // blow-up that Jacobi's relative accuracy does not, and on the exactly structured
  // Gram matrices of the transmon eigenbasis (rank-one 4 x 4) it hit its iteration
  // limit with a non-finite eigenvalue; the solver sweep on GB300 (qlb_eig_check)
  // has it no faster than Jacobi above n = 8.  Planned sizes above 24: Jacobi over
  // a thread-block cluster (rows of G and V in distributed shared memory).
  if (e.n_max > 24 && e.n_max <= EIG_CL_MAX_NP) {
    if (e.n_max <= 128) return launch_eig_cl<R, 8>(e, d_dims, s, prof);
    return launch_eig_cl<R, 16>(e, d_dims, s, prof);
  }
  size_t want = eig_smem_bytes<R>(e.n_max);
  int dyn = (int)(want <= EIG_SMEM_LIMIT ? want : EIG_SMEM_LIMIT);
  // FP64: a few warps suffice (ncu shows the solve waiting on its round barriers
  // and the DFMA pipe, not on issue slots).  Double-float: long dependent FP32
  // chains per rotation, so a full CTA of warps hides their latency.
  constexpr bool wide = std::is_same<R, df64>::value;
  if (e.n_max <= 24)
    k_eig<R, 128><<<1, 128, dyn, s>>>(e, (int*)d_dims, (cx<R>*)work, dyn, prof, nullptr);
  else if (wide)
    k_eig<R, 1024><<<1, 1024, dyn, s>>>(e, (int*)d_dims, (cx<R>*)work, dyn, prof, nullptr);
  else
    k_eig<R, 512><<<1, 512, dyn, s>>>(e, (int*)d_dims, (cx<R>*)work, dyn, prof, nullptr);
  return cudaGetLastError();
}
template cudaError_t launch_eig<double>(const EigDesc&, const int*, cudaStream_t, void*, double*);
template cudaError_t launch_eig<df64>(const EigDesc&, const int*, cudaStream_t, void*, double*);

// The eigen-solves of S states in one launch, with the kernel launch_eig picks for
// the largest planned size n_max over the members (every kernel takes any runtime
// size up to its planned one): one CTA, or one cluster, per member (blockIdx.y).
template <typename R>
cudaError_t launch_eig_group(int n_max, const EigDesc* d_grp, int S, cudaStream_t s, double* prof) {
  if (S <= 0) return cudaSuccess;
  EigDesc e{};
  e.n_max = n_max;
  if (n_max > 24 && n_max <= EIG_CL_MAX_NP) {
    if (n_max <= 128) return launch_eig_cl<R, 8>(e, nullptr, s, prof, d_grp, S);
    return launch_eig_cl<R, 16>(e, nullptr, s, prof, d_grp, S);
  }
  size_t want = eig_smem_bytes<R>(n_max);
  int dyn = (int)(want <= EIG_SMEM_LIMIT ? want : EIG_SMEM_LIMIT);
  constexpr bool wide = std::is_same<R, df64>::value;
  if (n_max <= 24)
    k_eig<R, 128, true><<<dim3(1, S), 128, dyn, s>>>(e, nullptr, nullptr, dyn, prof, d_grp);
  else if (wide)
    k_eig<R, 1024, true><<<dim3(1, S), 1024, dyn, s>>>(e, nullptr, nullptr, dyn, prof, d_grp);
  else
    k_eig<R, 512, true><<<dim3(1, S), 512, dyn, s>>>(e, nullptr, nullptr, dyn, prof, d_grp);
  return cudaGetLastError();
}
template cudaError_t launch_eig_group<double>(int, const EigDesc*, int, cudaStream_t, double*);
template cudaError_t launch_eig_group<df64>(int, const EigDesc*, int, cudaStream_t, double*);

// One named solver regardless of the size rule above (the check entry point):
// 1 one-CTA Jacobi, 2 cluster Jacobi over 8 CTAs (n <= 128), 3 over 16 CTAs
// (n <= 256), 4 Householder + QL (FP64, n <= 64).
template <typename R>
cudaError_t launch_eig_kind(int kind, const EigDesc& e, const int* d_dims, cudaStream_t s, void* work,
                            double* prof) {
  if (kind == 2 && e.n_max <= 128) return launch_eig_cl<R, 8>(e, d_dims, s, prof);
  if (kind == 3 && e.n_max <= EIG_CL_MAX_NP) return launch_eig_cl<R, 16>(e, d_dims, s, prof);
  if (kind == 4 && std::is_same<R, double>::value && e.n_max <= HEEV_N_MAX) {
    size_t want = eig_smem_bytes<double>(e.n_max);
    int dyn = (int)(want <= HEEV_SMEM_LIMIT ? want : HEEV_SMEM_LIMIT);
    k_heev<128><<<1, 128, dyn, s>>>(e, (int*)d_dims, (zd*)work, dyn, prof);
    return cudaGetLastError();
  }
  if (kind == 1) {
    size_t want = eig_smem_bytes<R>(e.n_max);
    int dyn = (int)(want <= EIG_SMEM_LIMIT ? want : EIG_SMEM_LIMIT);
    if (e.n_max <= 24)
      k_eig<R, 128><<<1, 128, dyn, s>>>(e, (int*)d_dims, (cx<R>*)work, dyn, prof, nullptr);
    else if (std::is_same<R, df64>::value)
      k_eig<R, 1024><<<1, 1024, dyn, s>>>(e, (int*)d_dims, (cx<R>*)work, dyn, prof, nullptr);
    else
      k_eig<R, 512><<<1, 512, dyn, s>>>(e, (int*)d_dims, (cx<R>*)work, dyn, prof, nullptr);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}
template cudaError_t launch_eig_kind<double>(int, const EigDesc&, const int*, cudaStream_t, void*, double*);
template cudaError_t launch_eig_kind<df64>(int, const EigDesc&, const int*, cudaStream_t, void*, double*);

void init_kernel_attributes() {
  cudaFuncSetAttribute(k_eig<double, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_LIMIT);
  cudaFuncSetAttribute(k_eig<double, 512, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_LIMIT);
  cudaFuncSetAttribute(k_eig<df64, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_LIMIT);
  cudaFuncSetAttribute(k_eig<df64, 1024, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_LIMIT);
  cudaFuncSetAttribute(k_eig_cl<double, 256, 8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)EIG_SMEM_LIMIT);
  cudaFuncSetAttribute(k_eig_cl<double, 256, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)EIG_SMEM_LIMIT);
  cudaFuncSetAttribute(k_eig_cl<double, 256, 16, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(k_eig_cl<df64, 256, 8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_LIMIT);
  cudaFuncSetAttribute(k_eig_cl<df64, 256, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)EIG_SMEM_LIMIT);
  cudaFuncSetAttribute(k_eig_cl<df64, 256, 16, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  set_attr<double, 128>();
  set_attr<double, 256>();
  set_attr<double, 512>();
  set_attr<df64, 128>();
  set_attr<df64, 256>();
  set_attr<df64, 512>();
  set_attr<df64, 1024>();
  cudaFuncSetAttribute(k_heev<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HEEV_SMEM_LIMIT);
  cudaFuncSetAttribute(k_eig_cl<double, 256, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_LIMIT);
  cudaFuncSetAttribute(k_eig_cl<double, 256, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_LIMIT);
  cudaFuncSetAttribute(k_eig_cl<double, 256, 16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(k_eig_cl<df64, 256, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_LIMIT);
  cudaFuncSetAttribute(k_eig_cl<df64, 256, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_LIMIT);
  cudaFuncSetAttribute(k_eig_cl<df64, 256, 16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

}  // namespace qlb
