// Range basis of a zip-up bond without an eigen-solve.
//
// The zip-up (Sec. III.A MPO.MPS product, Sec. V.A) cuts its bonds at a relative
// weight tol * zip_tol_factor, far below the final truncation: it needs an
// orthonormal U (n x r) with || (1 - U U^dag) M ||_F^2 <= tol' ||M||_F^2, not the
// eigen-decomposition of G = M M^dag.  This kernel builds U by column-pivoted
// Gram-Schmidt on the columns of G, each new basis vector re-orthogonalised against
// the basis so far (classical Gram-Schmidt passes, a second one when the first
// cancels more than three quarters of the squared norm: "twice is enough",
// Giraud, Langou & Rozloznik 2005).
//
// With W = (1 - Q Q^dag) G the residual of G's columns after j basis vectors,
// the discarded weight is Tr((1 - Q Q^dag) G) = sum_k Re W_kk, and the columns
// already chosen contribute zero, so the weight is known exactly at every step
// from the diagonal of the columns still open.  Step j:
//   (a) stop with r = j when that weight <= tol * Tr G;
//   (b) stop with r = j when the largest residual column norm, or that column's
//       residual after re-orthogonalisation, is at the rounding level of the
//       working precision (<= eps ||G||_F): only rounding is left;
//   (c) at j = cap the cut would drop real weight: the best rank-cap subspace is
//       the top eigenvectors of G, so the kernel sets the gate and leaves the bond
//       to the Jacobi solve launched behind it (which runs only when gated in);
//   else the column p with the largest residual norm becomes
//       q_j = normalise((1 - Q Q^dag) w_p)
//   and every open column k loses its component: w_k -= q_j (q_j^dag w_k).
//
// One CTA of 512 threads.  W is column-major (column k contiguous) in shared
// memory when n^2 complex numbers fit, else in a global workspace; a chosen
// column's slot is overwritten by its basis vector.  The column sweeps give each
// column a group of 8 lanes; every reduction is a fixed shuffle tree followed by
// per-warp slots summed in warp order, so the result does not depend on timing.
//
// Instantiated for R = double (the FP64 form) and R = df64 (the mixed forms).
// G and U are FP64 in both.

#include "builder.cuh"
#include "df64.cuh"

namespace qlb {

namespace {

template <typename R>
struct QrEps;
template <>
struct QrEps<double> {
  static constexpr double v = 2.220446049250313e-16;
};
template <>
struct QrEps<df64> {
  static constexpr double v = 3.552713678800501e-15;  // 2^-48
};

constexpr int QR_NT = 512;
constexpr int QR_WARPS = QR_NT / 32;
constexpr int QR_LG = 8;               // lanes per column in the column sweeps
constexpr int QR_NG = QR_NT / QR_LG;   // column groups
constexpr int QR_MAX_N = 512;
constexpr size_t QR_SMEM_LIMIT = 200 * 1024;

__device__ __forceinline__ double shx(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ df64 shx(df64 v, int m) {
  return df64(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}
template <typename R>
__device__ __forceinline__ cx<R> shx(cx<R> v, int m) {
  return mk<R>(shx(v.re, m), shx(v.im, m));
}
// sum over the 8 lanes of a column group (every lane of the group gets it)
template <typename T>
__device__ __forceinline__ T group_sum(T v) {
  v = v + shx(v, 1);
  v = v + shx(v, 2);
  v = v + shx(v, 4);
  return v;
}
template <typename R>
__device__ __forceinline__ cx<R> group_sum(cx<R> v) {
  return mk<R>(group_sum(v.re), group_sum(v.im));
}
// a small constant in the working type without an FP64 conversion
template <typename R>
__device__ __forceinline__ R rc(float x);
template <>
__device__ __forceinline__ double rc<double>(float x) {
  return (double)x;
}
template <>
__device__ __forceinline__ df64 rc<df64>(float x) {
  return df64(x, 0.f);
}
// c + a * b as one fused step: an FMA in FP64, a multiply-add with one
// renormalisation in double-float (about half the FP32 instructions of a separate
// double-float product and sum, at the same ~2^-44 relative accuracy)
__device__ __forceinline__ double qmac(double c, double a, double b) { return fma(a, b, c); }
__device__ __forceinline__ df64 qmac(df64 c, df64 a, df64 b) { return df_mac(c, a, b); }
// acc += conj(q) * w
template <typename R>
__device__ __forceinline__ void cdot_acc(cx<R>& acc, cx<R> q, cx<R> w) {
  acc.re = qmac(qmac(acc.re, q.re, w.re), q.im, w.im);
  acc.im = qmac(qmac(acc.im, q.re, w.im), -q.im, w.re);
}
// acc += q * a
template <typename R>
__device__ __forceinline__ void cmul_acc(cx<R>& acc, cx<R> q, cx<R> a) {
  acc.re = qmac(qmac(acc.re, q.re, a.re), -q.im, a.im);
  acc.im = qmac(qmac(acc.im, q.re, a.im), q.im, a.re);
}
// w - q * a
template <typename R>
__device__ __forceinline__ cx<R> csub_mul(cx<R> w, cx<R> q, cx<R> a) {
  w.re = qmac(qmac(w.re, -q.re, a.re), q.im, a.im);
  w.im = qmac(qmac(w.im, -q.re, a.im), -q.im, a.re);
  return w;
}
// nu + |w|^2
template <typename R>
__device__ __forceinline__ R abs2_acc(R nu, cx<R> w) {
  return qmac(qmac(nu, w.re, w.re), w.im, w.im);
}

// One sweep over the open columns: optionally w_k -= q (q^dag w_k); then the
// residual norm^2 and diagonal of every open column, reduced to the per-warp slots
// (largest norm with its column, ties to the lower index; sum of diagonals).  All
// in the working type: for double-float no instruction of the sweep uses the FP64
// pipe, which on this GPU retires ~2 operations per clock per SM.
template <typename R>
__device__ void column_sweep(cx<R>* W, int n, const cx<R>* q, const unsigned char* done, R* s_nu, int* s_k,
                             R* s_w) {
  const int tid = threadIdx.x, g = tid / QR_LG, gl = tid % QR_LG;
  const R zero = rc<R>(0.0f), minus1 = rc<R>(-1.0f);
  R best = minus1, wsum = zero;
  int bk = 0x7fffffff;
  for (int k0 = 0; k0 < n; k0 += QR_NG) {
    const int k = k0 + g;
    const bool act = k < n && !done[k];
    cx<R>* wk = W + (long)(act ? k : 0) * n;
    cx<R> a = mk<R>(zero, zero);
    if (q) {
      cx<R> part = mk<R>(zero, zero);
      if (act)
        for (int i = gl; i < n; i += QR_LG) cdot_acc(part, q[i], wk[i]);
      a = group_sum(part);
    }
    R nu = zero, dk = zero;
    if (act) {
      for (int i = gl; i < n; i += QR_LG) {
        cx<R> w = wk[i];
        if (q) {
          w = csub_mul(w, q[i], a);
          wk[i] = w;
        }
        nu = abs2_acc(nu, w);
        if (i == k) dk = w.re;
      }
    }
    nu = group_sum(nu);
    dk = group_sum(dk);
    if (act && gl == 0) {
      if (nu > best || (nu == best && k < bk)) {
        best = nu;
        bk = k;
      }
      wsum = wsum + dk;
    }
  }
  for (int o = QR_LG; o < 32; o <<= 1) {
    const R ob = shx(best, o);
    const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
    const R ow = shx(wsum, o);
    if (ob > best || (ob == best && ok < bk)) {
      best = ob;
      bk = ok;
    }
    wsum = wsum + ow;
  }
  if ((tid & 31) == 0) {
    s_nu[tid >> 5] = best;
    s_k[tid >> 5] = bk;
    s_w[tid >> 5] = wsum;
  }
}

// sum of a value over the CTA, the same in every thread (shuffle tree, then the
// per-warp slots in warp order); one barrier
template <typename R>
__device__ __forceinline__ R cta_sum(R v, R* slot) {
  for (int o = 16; o > 0; o >>= 1) v = v + shx(v, o);
  if ((threadIdx.x & 31) == 0) slot[threadIdx.x >> 5] = v;
  __syncthreads();
  R s = slot[0];
  for (int w = 1; w < QR_WARPS; w++) s = s + slot[w];
  return s;
}

template <typename R, bool GRP = false>
__global__ void __launch_bounds__(QR_NT) k_zipqr(EigDesc e, int* __restrict__ d, cx<R>* work, int dyn_bytes,
                                                  double* prof, const EigDesc* __restrict__ grp) {
  extern __shared__ unsigned char smem_raw[];
  if constexpr (GRP) {  // grouped launch: one CTA per member (blockIdx.y)
    e = grp[blockIdx.y];
    d = e.dims;
    work = (cx<R>*)e.work;
  }
  __shared__ cx<R> s_c[QR_MAX_N];       // re-orthogonalisation coefficients q_i^dag w_p
  __shared__ cx<R> s_part[QR_NT];       // partial sums of sum_i c_i q_i[row]
  __shared__ int s_q[QR_MAX_N];         // column slot of q_j
  __shared__ unsigned char s_done[QR_MAX_N];
  __shared__ R s_nu[QR_WARPS], s_w[QR_WARPS], s_r[3][QR_WARPS];
  __shared__ int s_k[QR_WARPS];
  const int n = dev_eval(e.n, d);
  const int tid = threadIdx.x, g = tid / QR_LG, gl = tid % QR_LG;
  const R zero = rc<R>(0.0f);
  if (n <= 0 || n > QR_MAX_N) {
    if (tid == 0) {
      if (n > QR_MAX_N && e.err) atomicOr(e.err, 2);
      d[e.dim_out] = n <= 0 ? 0 : 1;
      if (e.gate) *e.gate = n > QR_MAX_N ? 1 : 0;
    }
    return;
  }
  cx<R>* W = (size_t)n * n * sizeof(cx<R>) <= (size_t)dyn_bytes ? (cx<R>*)smem_raw : work;
  const zd* G = (const zd*)e.G;
  // W = G column by column: column k of a Hermitian G is the conjugate of row k
  R tr = zero, fr = zero;
  for (long x = tid; x < (long)n * n; x += QR_NT) {
    const int k = (int)(x / n), i = (int)(x - (long)k * n);
    const zd v = G[x];
    const cx<R> w = mk<R>(R(v.re), R(i == k ? 0.0 : -v.im));
    W[x] = w;
    fr = abs2_acc(fr, w);
    if (i == k) tr = tr + w.re;
  }
  for (int i = tid; i < n; i += QR_NT) s_done[i] = 0;
  tr = cta_sum(tr, s_r[0]);
  fr = cta_sum(fr, s_r[1]);
  const bool finite = isfinite(tr) && isfinite(fr);
  int cap = dev_eval(e.cap, d);
  if (cap < 1) cap = 1;
  // thresholds of the stop tests, as squared norms in the working type
  const R thr_w = R(e.tol) * tr;
  const R floor2 = R(QrEps<R>::v * QrEps<R>::v) * fr;
  const R quarter = rc<R>(0.25f);
  const int npad = (n + 31) & ~31;
  const int S = QR_NT / npad;  // n <= 512, so S >= 1
  double flops = 0.0;          // thread 0 only

  int j = 0, nred = 0;
  bool fallback = false;
  if (finite) {
    column_sweep<R>(W, n, nullptr, s_done, s_nu, s_k, s_w);
    __syncthreads();
    for (;; j++) {
      // every thread reduces the per-warp slots in the same order
      R best = rc<R>(-1.0f), wres = zero;
      int p = 0x7fffffff;
      for (int w = 0; w < QR_WARPS; w++) {
        const R b = s_nu[w];
        const int k = s_k[w];
        if (b > best || (b == best && k < p)) {
          best = b;
          p = k;
        }
        wres = wres + s_w[w];
      }
      if (j == n || p >= n) break;  // p >= n: no open column compared (non-finite norms)
      if (j >= 1 && (wres <= thr_w || best <= floor2)) break;
      if (j >= cap) {
        fallback = true;
        break;
      }
      cx<R>* wp = W + (long)p * n;
      const int row = tid % npad, part = tid / npad;
      cx<R> v = mk<R>(zero, zero);
      if (part == 0 && row < n) v = wp[row];
      R nrm2 = best;
      // the pivot column projected against the basis so far once more, and a third
      // time when a pass removes more than three quarters of its squared norm
      // (Kahan-Parlett "twice is enough": the second projection leaves rounding of
      // the first only when little cancels)
      for (int pass = 0; j > 0 && pass < 2; pass++) {
        // c_i = q_i^dag w_p, one column group per i
        for (int i0 = 0; i0 < j; i0 += QR_NG) {
          const int i = i0 + g;
          cx<R> acc = mk<R>(zero, zero);
          if (i < j) {
            const cx<R>* qi = W + (long)s_q[i] * n;
            for (int r = gl; r < n; r += QR_LG) cdot_acc(acc, qi[r], wp[r]);
          }
          acc = group_sum(acc);
          if (i < j && gl == 0) s_c[i] = acc;
        }
        __syncthreads();
        // partial sums of sum_i c_i q_i[row] over i = part (mod S)
        if (part < S && row < n) {
          cx<R> acc = mk<R>(zero, zero);
          for (int i = part; i < j; i += S) cmul_acc(acc, s_c[i], W[(long)s_q[i] * n + row]);
          s_part[part * npad + row] = acc;
        }
        __syncthreads();
        if (part == 0 && row < n) {
          v = wp[row];
          for (int s2 = 0; s2 < S; s2++) v = csub(v, s_part[s2 * npad + row]);
          wp[row] = v;
        }
        const R prev = nrm2;
        // three slot sets in rotation: a set is written again only two barriers later
        nrm2 = cta_sum((part == 0 && row < n) ? cabs2(v) : zero, s_r[nred++ % 3]);
        if (tid == 0) flops += 16.0 * n * j;
        if (nrm2 >= quarter * prev) break;
      }
      // the pivot's true residual is at the rounding level: what the tracked norms
      // still show is rounding of earlier projections, and the range is complete
      if (j >= 1 && nrm2 <= floor2) break;
      if (part == 0 && row < n) {
        cx<R> qv;
        if (nrm2 > zero) {
          const R inv = rc<R>(1.0f) / sqrt(nrm2);
          qv = mk<R>(v.re * inv, v.im * inv);
        } else {
          qv = mk<R>(rc<R>(row == p ? 1.0f : 0.0f), zero);  // G = 0: any unit vector spans it
        }
        wp[row] = qv;
      }
      if (tid == 0) {
        s_done[p] = 1;
        s_q[j] = p;
      }
      __syncthreads();
      column_sweep<R>(W, n, wp, s_done, s_nu, s_k, s_w);
      if (tid == 0) flops += 20.0 * n * (n - j - 1);
      __syncthreads();
    }
  }
  const int r = finite ? j : 1;
  if (fallback) {
    if (tid == 0) {
      if (e.gate) *e.gate = 1;
      if (e.solver_stats) {
        atomicAdd(e.solver_stats + 7, 1.0);
        atomicAdd(e.solver_stats + 8, 1.0);
      }
      if (prof) atomicAdd(prof, flops);
    }
    return;
  }
  if (tid == 0) {
    d[e.dim_out] = r;
    if (e.gate) *e.gate = 0;
    if (!finite && e.err) atomicOr(e.err, 2);
    if (e.solver_stats) {
      atomicAdd(e.solver_stats + 0, 1.0);
      atomicAdd(e.solver_stats + 2, (double)n);
      atomicAdd(e.solver_stats + 3, (double)r);
      atomicAdd(e.solver_stats + 7, 1.0);
      atomicMax((unsigned long long*)(e.solver_stats + 6), (unsigned long long)__double_as_longlong((double)n));
    }
    if (prof) {
      atomicAdd(prof, flops);
      atomicAdd(prof + QLB_K_COUNT, sizeof(zd) * ((double)n * n + (double)n * r));
    }
  }
  zd* out = (zd*)e.out;
  for (long x = tid; x < (long)n * r; x += QR_NT) {
    cx<R> u;
    int i, jj;
    if (e.out_mode == 0) {
      i = (int)(x / r);
      jj = (int)(x - (long)i * r);
    } else {
      jj = (int)(x / n);
      i = (int)(x - (long)jj * n);
    }
    if (finite)
      u = W[(long)s_q[jj] * n + i];
    else
      u = mk<R>(rc<R>(i == 0 ? 1.0f : 0.0f), zero);
    if (e.out_mode == 0)
      out[x] = mk<double>((double)u.re, (double)u.im);
    else if (e.out_mode == 1)
      out[x] = mk<double>((double)u.re, -(double)u.im);
  }
}

}  // namespace

size_t zipqr_workspace_elems(int n_max) {
  const size_t need = (size_t)n_max * n_max;
  return need * sizeof(zd) > QR_SMEM_LIMIT ? need : 1;
}

template <typename R>
cudaError_t launch_zipqr(const EigDesc& e, const int* d_dims, cudaStream_t s, void* work, double* prof) {
  const size_t want = (size_t)e.n_max * e.n_max * sizeof(cx<R>);
  const int dyn = (int)(want <= QR_SMEM_LIMIT ? want : QR_SMEM_LIMIT);
  k_zipqr<R><<<1, QR_NT, dyn, s>>>(e, (int*)d_dims, (cx<R>*)work, dyn, prof, nullptr);
  return cudaGetLastError();
}
template cudaError_t launch_zipqr<double>(const EigDesc&, const int*, cudaStream_t, void*, double*);
template cudaError_t launch_zipqr<df64>(const EigDesc&, const int*, cudaStream_t, void*, double*);

// The range bases of S states' zip-up bonds in one launch (one CTA per member);
// n_max is the largest planned size over the members.
template <typename R>
cudaError_t launch_zipqr_group(int n_max, const EigDesc* d_grp, int S, cudaStream_t s, double* prof) {
  if (S <= 0) return cudaSuccess;
  const size_t want = (size_t)n_max * n_max * sizeof(cx<R>);
  const int dyn = (int)(want <= QR_SMEM_LIMIT ? want : QR_SMEM_LIMIT);
  EigDesc dummy{};
  k_zipqr<R, true><<<dim3(1, S), QR_NT, dyn, s>>>(dummy, nullptr, nullptr, dyn, prof, d_grp);
  return cudaGetLastError();
}
template cudaError_t launch_zipqr_group<double>(int, const EigDesc*, int, cudaStream_t, double*);
template cudaError_t launch_zipqr_group<df64>(int, const EigDesc*, int, cudaStream_t, double*);

cudaError_t launch_solver(bool mixed, int solver, const EigDesc& e, const int* d_dims, cudaStream_t s, void* work) {
  if (solver == 5)
    return mixed ? launch_zipqr<df64>(e, d_dims, s, work, nullptr) : launch_zipqr<double>(e, d_dims, s, work, nullptr);
  if (solver == 0)
    return mixed ? launch_eig<df64>(e, d_dims, s, work, nullptr) : launch_eig<double>(e, d_dims, s, work, nullptr);
  return mixed ? launch_eig_kind<df64>(solver, e, d_dims, s, work, nullptr)
               : launch_eig_kind<double>(solver, e, d_dims, s, work, nullptr);
}

void init_qr_attributes() {
  cudaFuncSetAttribute(k_zipqr<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)QR_SMEM_LIMIT);
  cudaFuncSetAttribute(k_zipqr<df64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)QR_SMEM_LIMIT);
  cudaFuncSetAttribute(k_zipqr<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)QR_SMEM_LIMIT);
  cudaFuncSetAttribute(k_zipqr<df64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)QR_SMEM_LIMIT);
}

}  // namespace qlb
