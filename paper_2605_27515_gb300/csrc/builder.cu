// Quantics MPO builder (Sec. II.B): dense per-mode operators -> TT-SVD -> MPO,
// MPO sums (block stacking) and recompression, all on the device.
//
// The SVD used here is the one-sided (Hestenes) Jacobi method on the rows of the
// matrix: pairs of rows are rotated until every pair is orthogonal to working
// precision.  Unlike an eigen-solve of the Gram matrix it resolves small singular
// values to high relative accuracy, which the exact operator ranks of Table I need.
// It runs at setup only, always in FP64.

#include <algorithm>
#include <cmath>
#include <cstring>

#include "builder.cuh"

namespace qlb {

// ------------------------------------------------------------------ memory

qlb_status dev_alloc(qlb_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (ctx->opt.hbm_budget && ctx->mem_held + bytes > ctx->opt.hbm_budget) {
    set_error("device memory budget exceeded (" + std::to_string(ctx->mem_held + bytes) + " > " +
              std::to_string(ctx->opt.hbm_budget) + " bytes)");
    return QLB_ENOMEM;
  }
  // Stream-ordered allocation from the device's memory pool: unlike cudaMalloc /
  // cudaFree it never synchronises the whole device, so admitting or retiring one
  // state does not drain the steps other states have in flight.  The buffer is
  // complete when the context stream is, which the synchronisation below ensures
  // before any other stream touches it.
  cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error(std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    return QLB_ENOMEM;
  }
  ctx->mem_held += bytes;
  ctx->n_allocs++;
  g_alloc_sizes()[*p] = std::make_pair(bytes, ctx);
  return QLB_OK;
}

// Returns p to the pool in the order of its owner's stream (every caller has
// synchronised the streams that used p); without a live owner, plain cudaFree.
void dev_free(qlb_ctx*, void* p) {
  if (!p) return;
  auto& m = g_alloc_sizes();
  auto it = m.find(p);
  qlb_ctx* owner = nullptr;
  if (it != m.end()) {
    owner = it->second.second;
    if (owner) owner->mem_held -= std::min(owner->mem_held, it->second.first);
    m.erase(it);
  }
  if (owner && owner->stream)
    cudaFreeAsync(p, owner->stream);
  else
    cudaFree(p);
}

std::map<void*, std::pair<size_t, qlb_ctx*>>& g_alloc_sizes() {
  static std::map<void*, std::pair<size_t, qlb_ctx*>> m;
  return m;
}

namespace {

constexpr int B_THREADS = 256;

__device__ __forceinline__ int rr_player_b(int pos, int round, int np) {
  if (pos == 0) return 0;
  return 1 + (pos - 1 + round) % (np - 1);
}

template <typename T>
__device__ T block_sum(T v, T* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  T r = 0;
  if (threadIdx.x < (blockDim.x >> 5)) r = sh[threadIdx.x];
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  __syncthreads();
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// One round of row-wise one-sided Jacobi: block t rotates the pair of rows that
// round-robin position t holds in this round.  X is m x n (ld n), T is m x m.
// A pair is rotated only when |<x_p, x_q>| exceeds both ~sqrt(n) eps |x_p| |x_q|
// (relative orthogonality) and abs_thr = 1e-31 ||X||_F^2: without the absolute floor, the
// excess rows of a rank-deficient matrix keep rotating rounding noise forever.
__global__ void __launch_bounds__(B_THREADS) k_osj_round(zd* X, int m, int n, zd* T, int np, int round, int* cnt,
                                                        const double* abs_thr) {
  __shared__ double sh[32];
  __shared__ double s_c;
  __shared__ zd s_sp;
  __shared__ int s_rot;
  int t = blockIdx.x;
  int p = rr_player_b(t, round, np), q = rr_player_b(np - 1 - t, round, np);
  if (p > q) {
    int x = p;
    p = q;
    q = x;
  }
  if (q >= m) return;
  zd* xp = X + (long)p * n;
  zd* xq = X + (long)q * n;
  double a = 0, b = 0, gr = 0, gi = 0;
  for (int j = threadIdx.x; j < n; j += B_THREADS) {
    zd u = xp[j], v = xq[j];
    a += u.re * u.re + u.im * u.im;
    b += v.re * v.re + v.im * v.im;
    // u * conj(v)
    gr += u.re * v.re + u.im * v.im;
    gi += u.im * v.re - u.re * v.im;
  }
  a = block_sum(a, sh);
  b = block_sum(b, sh);
  gr = block_sum(gr, sh);
  gi = block_sum(gi, sh);
  if (threadIdx.x == 0) {
    double x = sqrt(gr * gr + gi * gi);
    s_rot = 0;
    // relative floor: a length-n dot product carries ~sqrt(n) eps of rounding
    double rel = 2.220446049250313e-16 * fmax(8.0, 4.0 * sqrt((double)n));
    if (x > 0.0 && x > rel * sqrt(a * b) && x > *abs_thr) {
      double tau = (b - a) / (2 * x);
      double tt = fabs(tau) > 1e100 ? 0.5 / tau : (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      double c = 1.0 / sqrt(1.0 + tt * tt);
      double s = tt * c;
      s_c = c;
      s_sp = mk<double>(s * gr / x, s * gi / x);
      s_rot = 1;
      atomicAdd(cnt, 1);
    }
  }
  __syncthreads();
  if (!s_rot) return;
  double c = s_c;
  zd sp = s_sp;
  for (int j = threadIdx.x; j < n; j += B_THREADS) {
    zd u = xp[j], v = xq[j];
    xp[j] = csub(cscale(u, c), cmul(sp, v));
    xq[j] = cadd(cmul(cconj(sp), u), cscale(v, c));
  }
  zd* tp = T + (long)p * m;
  zd* tq = T + (long)q * m;
  for (int j = threadIdx.x; j < m; j += B_THREADS) {
    zd u = tp[j], v = tq[j];
    tp[j] = csub(cscale(u, c), cmul(sp, v));
    tq[j] = cadd(cmul(cconj(sp), u), cscale(v, c));
  }
}

// All sweeps of the row-wise one-sided Jacobi in one CTA (for moderate sizes):
// warp w rotates the pairs w, w + 32, ... of each round; rounds are separated by
// __syncthreads().  Stops after a sweep without rotation or after max_sweeps;
// writes the number of sweeps run, or -1 when it stopped at the limit.
constexpr int OSJ1_THREADS = 1024;
__global__ void __launch_bounds__(OSJ1_THREADS) k_osj_all(zd* X, int m, int n, zd* T, const double* abs_thr_p,
                                                        int max_sweeps, int* sweeps_out) {
  __shared__ int s_rot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = OSJ1_THREADS >> 5;
  const int np = m + (m & 1);
  const double abs_thr = *abs_thr_p;
  const double rel = 2.220446049250313e-16 * fmax(8.0, 4.0 * sqrt((double)n));
  int sw = 0;
  for (; sw < max_sweeps; sw++) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; round++) {
      for (int t = warp; t < np / 2; t += nwarps) {
        int p = rr_player_b(t, round, np), q = rr_player_b(np - 1 - t, round, np);
        if (p > q) {
          int x = p;
          p = q;
          q = x;
        }
        if (q >= m) continue;
        zd* xp = X + (long)p * n;
        zd* xq = X + (long)q * n;
        double a = 0, b = 0, gr = 0, gi = 0;
        for (int j = lane; j < n; j += 32) {
          zd u = xp[j], v = xq[j];
          a += u.re * u.re + u.im * u.im;
          b += v.re * v.re + v.im * v.im;
          gr += u.re * v.re + u.im * v.im;
          gi += u.im * v.re - u.re * v.im;
        }
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          gr += __shfl_xor_sync(0xffffffffu, gr, o);
          gi += __shfl_xor_sync(0xffffffffu, gi, o);
        }
        double x = sqrt(gr * gr + gi * gi);
        if (!(x > 0.0 && x > rel * sqrt(a * b) && x > abs_thr)) continue;
        double tau = (b - a) / (2 * x);
        double tt = fabs(tau) > 1e100 ? 0.5 / tau : (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + tt * tt);
        double s = tt * c;
        zd sp = mk<double>(s * gr / x, s * gi / x);
        for (int j = lane; j < n; j += 32) {
          zd u = xp[j], v = xq[j];
          xp[j] = csub(cscale(u, c), cmul(sp, v));
          xq[j] = cadd(cmul(cconj(sp), u), cscale(v, c));
        }
        zd* tp = T + (long)p * m;
        zd* tq = T + (long)q * m;
        for (int j = lane; j < m; j += 32) {
          zd u = tp[j], v = tq[j];
          tp[j] = csub(cscale(u, c), cmul(sp, v));
          tq[j] = cadd(cmul(cconj(sp), u), cscale(v, c));
        }
        if (lane == 0) atomicAdd(&s_rot, 1);
      }
      __syncthreads();
    }
    int nr = s_rot;
    __syncthreads();
    if (nr == 0) break;
  }
  if (threadIdx.x == 0) *sweeps_out = (sw < max_sweeps) ? sw + 1 : -1;
}

__global__ void k_abs_thr(const zd* X, long n, double* out) {
  __shared__ double sh[32];
  double acc = 0;
  for (long x = threadIdx.x; x < n; x += blockDim.x) acc += cabs2(X[x]);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = 1e-31 * acc;
}

__global__ void k_identity(zd* T, int m) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < (long)m * m) T[i] = mk<double>((i / m) == (i % m) ? 1.0 : 0.0, 0.0);
}

// Row norms, sort, truncation rule, outputs.  One CTA; dynamic smem holds
// w[m] (double) and perm[m] (int).
__global__ void k_osj_finish(const zd* X, int m, int n, const zd* T, double tol, int cap, double gap, zd* U,
                             int u_scale, zd* Rr, int r_unscale, int* k_out, double* s2_out) {
  extern __shared__ unsigned char sm[];
  double* w = (double*)sm;
  double* ws = w + m;
  int* perm = (int*)(ws + m);
  __shared__ int s_k;
  {  // row norms, one warp per row
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < m; i += nw) {
      double acc = 0;
      for (int j = lane; j < n; j += 32) acc += cabs2(X[(long)i * n + j]);
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) w[i] = acc;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    int r = 0;
    for (int j = 0; j < m; j++)
      if (w[j] > w[i] || (w[j] == w[i] && j < i)) r++;
    perm[r] = i;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < m; r += blockDim.x) ws[r] = w[perm[r]];
  __syncthreads();
  if (threadIdx.x == 0) {
    // same rule as the step's truncation (relative discarded weight, cap, clusters)
    double total = 0;
    for (int i = 0; i < m; i++) total += ws[i];
    int k = m;
    if (!(total > 0)) {
      k = 1;
    } else {
      double tail = 0;
      while (k > 1 && tail + ws[k - 1] <= tol * total) {
        tail += ws[k - 1];
        k--;
      }
      if (cap > 0 && k > cap) k = cap;
      if (k < m && sqrt(ws[k]) >= (1.0 - gap) * sqrt(ws[k - 1])) {
        int j = k;
        while (j < m && (cap <= 0 || j < cap) && sqrt(ws[j]) >= (1.0 - gap) * sqrt(ws[j - 1])) j++;
        if (j < m && sqrt(ws[j]) >= (1.0 - gap) * sqrt(ws[j - 1])) {
          j = k;
          while (j > 1 && sqrt(ws[j]) >= (1.0 - gap) * sqrt(ws[j - 1])) j--;
        }
        k = j;
      }
      if (k < 1) k = 1;
    }
    s_k = k;
    *k_out = k;
    if (s2_out)
      for (int i = 0; i < k; i++) s2_out[i] = ws[i];
  }
  __syncthreads();
  int k = s_k;
  // U[i, j] = conj(T[perm_j, i]) * s_j^u_scale
  for (long x = threadIdx.x; x < (long)m * k; x += blockDim.x) {
    int i = (int)(x / k), j = (int)(x % k);
    zd v = cconj(T[(long)perm[j] * m + i]);
    if (u_scale) v = cscale(v, sqrt(ws[j]));
    U[x] = v;
  }
  // R[j, :] = X[perm_j, :] / s_j^r_unscale
  for (long x = threadIdx.x; x < (long)k * n; x += blockDim.x) {
    int j = (int)(x / n), c = (int)(x % n);
    zd v = X[(long)perm[j] * n + c];
    if (r_unscale) {
      double s = sqrt(ws[j]);
      v = (s > 0) ? cscale(v, 1.0 / s) : mk<double>(0, 0);
    }
    Rr[x] = v;
  }
}

// Built-in single-mode factors (Sec. II.B; charge basis Sec. VII).
__global__ void k_factor(zd* F, int N, int kind, double param) {
  long x = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (x >= (long)N * N) return;
  int i = (int)(x / N), j = (int)(x % N);
  double v = 0;
  switch (kind) {
    case QLB_F_ID:
      v = (i == j);
      break;
    case QLB_F_A:
      v = (j == i + 1) ? sqrt((double)j) : 0.0;
      break;
    case QLB_F_ADAG:
      v = (i == j + 1) ? sqrt((double)i) : 0.0;
      break;
    case QLB_F_NUM:
      v = (i == j) ? (double)i : 0.0;
      break;
    case QLB_F_PARITY:
      v = (i == j) ? ((i & 1) ? -1.0 : 1.0) : 0.0;
      break;
    case QLB_F_CHARGE:
      v = (i == j) ? (double)i - param : 0.0;
      break;
    case QLB_F_COSPHI:
      v = (j == i + 1 || i == j + 1) ? 0.5 : 0.0;
      break;
  }
  F[x] = mk<double>(v, 0.0);
}

// Dense N x N (N = 2^R) -> tensor in quantics order [(s'_1 s_1), ..., (s'_R s_R)].
__global__ void k_tt_reshape_op(const zd* O, int R, zd* T) {
  long N = 1L << R;
  long x = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (x >= N * N) return;
  long row = x / N, col = x % N;
  long idx = 0;
  for (int i = 0; i < R; i++) {
    int so = (row >> (R - 1 - i)) & 1, si = (col >> (R - 1 - i)) & 1;
    idx = idx * 4 + 2 * so + si;
  }
  T[idx] = O[x];
}

__global__ void k_scale(zd* p, long n, zd c) {
  long x = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (x < n) p[x] = cmul(p[x], c);
}

// Add a [Da][P][Db] block into a larger [DA][P][DB] core at offset (oa, ob).
__global__ void k_place_block(const zd* src, int Da, int P, int Db, zd* dst, int DA, int DB, int oa, int ob) {
  long x = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (x >= (long)Da * P * Db) return;
  int a = (int)(x / (P * Db)), r = (int)(x % (P * Db));
  int p = r / Db, b = r % Db;
  zd* o = dst + ((long)(a + oa) * P + p) * DB + (b + ob);
  *o = cadd(*o, src[x]);
}

__global__ void k_zero(zd* p, long n) {
  long x = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (x < n) p[x] = mk<double>(0, 0);
}

__global__ void k_conj_transpose(const zd* A, zd* B, int N) {
  long x = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (x >= (long)N * N) return;
  int i = (int)(x / N), j = (int)(x % N);
  B[(long)j * N + i] = cconj(A[x]);
}

__global__ void k_abs_rowsum_max(const zd* A, int N, double* out) {
  __shared__ double sh[32];
  double best = 0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double s = 0;
    for (int j = 0; j < N; j++) s += sqrt(cabs2(A[(long)i * N + j]));
    best = fmax(best, s);
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) r = fmax(r, sh[w]);
    *out = r;
  }
}

inline unsigned nblk(long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------------ SVD (one-sided Jacobi)

qlb_status svd_osj(qlb_ctx* ctx, zd* X, int m, int n, double tol, int cap, zd** U, int u_scale, zd** Rr,
                   int r_unscale, int* k_out, int max_sweeps) {
  cudaStream_t s = ctx->stream;
  *U = *Rr = nullptr;
  zd* T = nullptr;
  int* d_cnt = nullptr;
  int* d_k = nullptr;
  qlb_status st;
  if ((st = dev_alloc(ctx, (void**)&T, sizeof(zd) * (size_t)m * m))) return st;
  if ((st = dev_alloc(ctx, (void**)&d_cnt, 4 * sizeof(double)))) {
    dev_free(ctx, T);
    return st;
  }
  d_k = d_cnt + 1;
  double* d_thr = (double*)d_cnt + 1;
  k_identity<<<nblk((long)m * m), 256, 0, s>>>(T, m);
  k_abs_thr<<<1, 256, 0, s>>>(X, (long)m * n, d_thr);
  int np = m + (m & 1);
  bool conv = (m <= 1);
  if (!conv && (long)n <= 16384) {
    // moderate rows: every sweep in one launch
    int* d_sw = d_cnt;
    k_osj_all<<<1, OSJ1_THREADS, 0, s>>>(X, m, n, T, d_thr, max_sweeps, d_sw);
    int h_sw = 0;
    cudaMemcpyAsync(&h_sw, d_sw, sizeof(int), cudaMemcpyDeviceToHost, s);
    QLB_CUDA_TRY(cudaStreamSynchronize(s));
    conv = h_sw > 0;
    max_sweeps = 0;  // skip the multi-launch loop below
  }
  for (int sw = 0; sw < max_sweeps && !conv; sw++) {
    cudaMemsetAsync(d_cnt, 0, sizeof(int), s);
    for (int r = 0; r < np - 1; r++) k_osj_round<<<np / 2, B_THREADS, 0, s>>>(X, m, n, T, np, r, d_cnt, d_thr);
    int h_cnt = 0;
    cudaMemcpyAsync(&h_cnt, d_cnt, sizeof(int), cudaMemcpyDeviceToHost, s);
    QLB_CUDA_TRY(cudaStreamSynchronize(s));
    conv = (h_cnt == 0);
  }
  if (!conv) {
    dev_free(ctx, T);
    dev_free(ctx, d_cnt);
    set_error("one-sided Jacobi SVD did not converge");
    return QLB_ENOTCONV;
  }
  // outputs at most min(m, n) wide... allocate for m (k <= m)
  int kmax = m;
  if ((st = dev_alloc(ctx, (void**)U, sizeof(zd) * (size_t)m * kmax)) ||
      (st = dev_alloc(ctx, (void**)Rr, sizeof(zd) * (size_t)kmax * n))) {
    dev_free(ctx, T);
    dev_free(ctx, d_cnt);
    dev_free(ctx, *U);
    *U = nullptr;
    return st;
  }
  size_t sm = (size_t)m * (2 * sizeof(double) + sizeof(int));
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_osj_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_osj_finish<<<1, 256, sm, s>>>(X, m, n, T, tol, cap, 1e-10, *U, u_scale, *Rr, r_unscale, d_k, nullptr);
  int hk = 0;
  cudaMemcpyAsync(&hk, d_k, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  dev_free(ctx, T);
  dev_free(ctx, d_cnt);
  if (e != cudaSuccess) {
    set_error(std::string("svd finish: ") + cudaGetErrorString(e));
    return QLB_EDEVICE;
  }
  *k_out = hk;
  return QLB_OK;
}

// ------------------------------------------------------------------ MPOs

Mpo::~Mpo() {
  for (auto p : core) dev_free(nullptr, p);
}
size_t Mpo::bytes() const {
  size_t b = 0;
  for (int i = 0; i < L; i++) b += sizeof(zd) * (size_t)D[i] * 4 * D[i + 1];
  return b;
}

void mpo_clear(qlb_ctx* ctx, Mpo& W) {
  for (auto p : W.core) dev_free(ctx, p);
  W.core.clear();
  W.D.clear();
  W.L = 0;
}

// TT-SVD of a tensor in quantics order with physical dimension P per site (P = 4
// for operators, 2 for vectors).  T (device, P^L entries) is consumed.
qlb_status tt_svd(qlb_ctx* ctx, zd* T, int L, int P, double tol, int cap, std::vector<zd*>& cores,
                  std::vector<int>& D) {
  cores.assign(L, nullptr);
  D.assign(L + 1, 1);
  long rest = 1;
  for (int i = 0; i < L; i++) rest *= P;
  zd* cur = T;
  int r = 1;
  for (int i = 0; i < L - 1; i++) {
    int m = r * P;
    long n = rest / P;
    zd *U, *Rr;
    int k;
    qlb_status st = svd_osj(ctx, cur, m, (int)n, tol, cap, &U, 0, &Rr, 0, &k, 60);
    dev_free(ctx, cur);
    if (st) {
      // the caller's vector must not keep the freed cores (its owner frees them again)
      for (auto& p : cores) {
        dev_free(ctx, p);
        p = nullptr;
      }
      return st;
    }
    // U is m x m storage with k columns used: compact it into the core [r][P][k]
    // (U rows are (r, p) in that order since X rows were)
    cores[i] = U;  // row-major m x k (k columns)
    D[i + 1] = k;
    cur = Rr;  // k x n, row-major; the next X is (k*P) x (n/P) with the same storage
    r = k;
    rest = n;
  }
  cores[L - 1] = cur;  // r x P x 1
  D[L] = 1;
  return QLB_OK;
}

qlb_status make_identity_mpo(qlb_ctx* ctx, int R, Mpo& W) {
  W.L = R;
  W.D.assign(R + 1, 1);
  W.core.assign(R, nullptr);
  for (int i = 0; i < R; i++) {
    qlb_status st = dev_alloc(ctx, (void**)&W.core[i], 4 * sizeof(zd));
    if (st) return st;
    zd h[4] = {mk<double>(1, 0), mk<double>(0, 0), mk<double>(0, 0), mk<double>(1, 0)};
    QLB_CUDA_TRY(cudaMemcpyAsync(W.core[i], h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
  }
  QLB_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return QLB_OK;
}

// MPO of one dense N x N single-mode matrix (N = 2^R) by TT-SVD.
qlb_status mpo_from_dense(qlb_ctx* ctx, const zd* F, int R, double tol, int cap, Mpo& W) {
  long N = 1L << R;
  zd* T = nullptr;
  qlb_status st = dev_alloc(ctx, (void**)&T, sizeof(zd) * N * N);
  if (st) return st;
  k_tt_reshape_op<<<nblk(N * N), 256, 0, ctx->stream>>>(F, R, T);
  W.L = R;
  return tt_svd(ctx, T, R, 4, tol, cap, W.core, W.D);
}

// Appends the sites of B after those of A (product of operators on disjoint sites).
void mpo_concat(Mpo& A, Mpo& B) {
  if (A.L == 0) {
    A.L = B.L;
    A.D = B.D;
    A.core = B.core;
  } else {
    for (int i = 0; i < B.L; i++) A.core.push_back(B.core[i]);
    for (int i = 1; i <= B.L; i++) A.D.push_back(B.D[i]);
    A.L += B.L;
  }
  B.core.clear();
  B.D.clear();
  B.L = 0;
}

qlb_status mpo_scale(qlb_ctx* ctx, Mpo& W, zd c) {
  long n = (long)W.D[0] * 4 * W.D[1];
  k_scale<<<nblk(n), 256, 0, ctx->stream>>>(W.core[0], n, c);
  QLB_CUDA_TRY(cudaGetLastError());
  return QLB_OK;
}

qlb_status mpo_copy(qlb_ctx* ctx, const Mpo& A, Mpo& B) {
  mpo_clear(ctx, B);
  B.L = A.L;
  B.D = A.D;
  B.core.assign(A.L, nullptr);
  for (int i = 0; i < A.L; i++) {
    size_t b = sizeof(zd) * (size_t)A.D[i] * 4 * A.D[i + 1];
    qlb_status st = dev_alloc(ctx, (void**)&B.core[i], b);
    if (st) return st;
    QLB_CUDA_TRY(cudaMemcpyAsync(B.core[i], A.core[i], b, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  return QLB_OK;
}

// Stack MPOs: block-diagonal cores; core 0 of block j lands on left-boundary rows
// [row_off[j], row_off[j] + D_0(j)) (all blocks on row 0 for a plain sum).
qlb_status mpo_stack(qlb_ctx* ctx, const std::vector<const Mpo*>& parts, const std::vector<int>& row_off, int D0,
                     Mpo& out) {
  mpo_clear(ctx, out);
  int L = parts[0]->L;
  out.L = L;
  out.D.assign(L + 1, 0);
  out.D[0] = D0;
  out.D[L] = 1;
  for (int i = 1; i < L; i++)
    for (auto p : parts) out.D[i] += p->D[i];
  out.core.assign(L, nullptr);
  for (int i = 0; i < L; i++) {
    long n = (long)out.D[i] * 4 * out.D[i + 1];
    qlb_status st = dev_alloc(ctx, (void**)&out.core[i], sizeof(zd) * n);
    if (st) return st;
    k_zero<<<nblk(n), 256, 0, ctx->stream>>>(out.core[i], n);
    int oa = 0, ob = 0;
    for (size_t j = 0; j < parts.size(); j++) {
      const Mpo* p = parts[j];
      int Da = p->D[i], Db = p->D[i + 1];
      int a0 = (i == 0) ? row_off[j] : oa;
      int b0 = (i == L - 1) ? 0 : ob;
      long ne = (long)Da * 4 * Db;
      k_place_block<<<nblk(ne), 256, 0, ctx->stream>>>(p->core[i], Da, 4, Db, out.core[i], out.D[i], out.D[i + 1], a0,
                                                      b0);
      oa += Da;
      ob += Db;
    }
  }
  QLB_CUDA_TRY(cudaGetLastError());
  return QLB_OK;
}

// Recompression of an MPO (left boundary never truncated): left-canonical sweep
// with exact SVDs, then right-to-left truncated SVDs.
qlb_status mpo_compress(qlb_ctx* ctx, Mpo& W, double tol, int cap) {
  const int L = W.L;
  cudaStream_t s = ctx->stream;
  qlb_status st;
  for (int i = 0; i < L - 1; i++) {
    int m = W.D[i] * 4, n = W.D[i + 1];
    zd *U, *Rr;
    int k;
    if ((st = svd_osj(ctx, W.core[i], m, n, 1e-32, 0, &U, 0, &Rr, 0, &k, 60))) return st;
    dev_free(ctx, W.core[i]);
    W.core[i] = U;  // [D_i][4][k]
    // core_{i+1} <- Rr (k x n) * core_{i+1} (n x 4 D_{i+2})
    int n2 = 4 * W.D[i + 2];
    zd* nc;
    if ((st = dev_alloc(ctx, (void**)&nc, sizeof(zd) * (size_t)k * n2))) return st;
    GemmDesc g{};
    g.A = Rr;
    g.B = W.core[i + 1];
    g.C = nc;
    g.m = dconst(k);
    g.n = dconst(n2);
    g.k = dconst(n);
    g.lda = dconst(n);
    g.ldb = dconst(n2);
    g.ldc = dconst(n2);
    g.sA1 = g.sB1 = g.sC1 = g.sA2 = g.sB2 = g.sC2 = dconst(0);
    g.nb1 = g.nb2 = dconst(1);
    g.opA = g.opB = OP_N;
    g.alpha_re = 1;
    g.m_max = k;
    g.n_max = n2;
    g.nb_max = 1;
    QLB_CUDA_TRY(launch_gemm<double>(g, nullptr, s, nullptr));
    dev_free(ctx, W.core[i + 1]);
    dev_free(ctx, Rr);
    W.core[i + 1] = nc;
    W.D[i + 1] = k;
  }
  for (int i = L - 1; i >= 1; i--) {
    int m = W.D[i], n = 4 * W.D[i + 1];
    zd *US, *Vh;
    int k;
    if ((st = svd_osj(ctx, W.core[i], m, n, tol, cap, &US, 1, &Vh, 1, &k, 60))) return st;
    dev_free(ctx, W.core[i]);
    W.core[i] = Vh;  // [k][4][D_{i+1}]
    int m2 = W.D[i - 1] * 4;
    zd* nc;
    if ((st = dev_alloc(ctx, (void**)&nc, sizeof(zd) * (size_t)m2 * k))) return st;
    GemmDesc g{};
    g.A = W.core[i - 1];
    g.B = US;
    g.C = nc;
    g.m = dconst(m2);
    g.n = dconst(k);
    g.k = dconst(m);
    g.lda = dconst(m);
    g.ldb = dconst(k);
    g.ldc = dconst(k);
    g.sA1 = g.sB1 = g.sC1 = g.sA2 = g.sB2 = g.sC2 = dconst(0);
    g.nb1 = g.nb2 = dconst(1);
    g.opA = g.opB = OP_N;
    g.alpha_re = 1;
    g.m_max = m2;
    g.n_max = k;
    g.nb_max = 1;
    QLB_CUDA_TRY(launch_gemm<double>(g, nullptr, s, nullptr));
    dev_free(ctx, W.core[i - 1]);
    dev_free(ctx, US);
    W.core[i - 1] = nc;
    W.D[i] = k;
  }
  QLB_CUDA_TRY(cudaStreamSynchronize(s));
  return QLB_OK;
}

// ------------------------------------------------------------------ operators

qlb_status make_factor(qlb_ctx* ctx, int N, const qlb_factor& f, zd** out) {
  qlb_status st = dev_alloc(ctx, (void**)out, sizeof(zd) * (size_t)N * N);
  if (st) return st;
  if (f.kind == QLB_F_DENSE) {
    if (!f.dense) {
      set_error("QLB_F_DENSE factor without a matrix");
      return QLB_EINVAL;
    }
    QLB_CUDA_TRY(cudaMemcpyAsync(*out, f.dense, sizeof(zd) * (size_t)N * N, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    if (f.kind < QLB_F_ID || f.kind > QLB_F_COSPHI) {
      set_error("unknown factor kind " + std::to_string(f.kind));
      return QLB_EINVAL;
    }
    k_factor<<<nblk((long)N * N), 256, 0, ctx->stream>>>(*out, N, f.kind, f.param);
  }
  QLB_CUDA_TRY(cudaGetLastError());
  return QLB_OK;
}

qlb_status dense_mul(qlb_ctx* ctx, const zd* A, int opA, const zd* B, int N, zd** out) {
  qlb_status st = dev_alloc(ctx, (void**)out, sizeof(zd) * (size_t)N * N);
  if (st) return st;
  GemmDesc g{};
  g.A = A;
  g.B = B;
  g.C = *out;
  g.m = g.n = g.k = dconst(N);
  g.lda = g.ldb = g.ldc = dconst(N);
  g.sA1 = g.sB1 = g.sC1 = g.sA2 = g.sB2 = g.sC2 = dconst(0);
  g.nb1 = g.nb2 = dconst(1);
  g.opA = opA;
  g.opB = OP_N;
  g.alpha_re = 1;
  g.m_max = g.n_max = N;
  g.nb_max = 1;
  QLB_CUDA_TRY(launch_gemm<double>(g, nullptr, ctx->stream, nullptr));
  return QLB_OK;
}

double dense_inf_norm(qlb_ctx* ctx, const zd* A, int N) {
  double* d = nullptr;
  if (dev_alloc(ctx, (void**)&d, sizeof(double))) return INFINITY;
  k_abs_rowsum_max<<<1, 256, 0, ctx->stream>>>(A, N, d);
  double h = INFINITY;
  cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  dev_free(ctx, d);
  return h;
}

// MPO of sum_t coeff_t (x)_m F_{t,m}; terms are summed one at a time with a
// recompression after each addition to keep the bond dimensions small.
qlb_status mpo_from_terms(qlb_system* sys, const std::vector<DevTerm>& terms, double tol, int cap, Mpo& out) {
  qlb_ctx* ctx = sys->ctx;
  mpo_clear(ctx, out);
  qlb_status st;
  for (size_t t = 0; t < terms.size(); t++) {
    Mpo term;
    for (int m = 0; m < sys->M; m++) {
      Mpo part;
      const std::string key = (terms[t].fac[m] && m < (int)terms[t].key.size() && !terms[t].key[m].empty())
                                  ? std::to_string(sys->R[m]) + "|" + terms[t].key[m]
                                  : std::string();
      auto hit = key.empty() ? ctx->factor_mpo_cache.end() : ctx->factor_mpo_cache.find(key);
      if (hit != ctx->factor_mpo_cache.end()) {
        st = mpo_copy(ctx, *hit->second, part);
      } else if (terms[t].fac[m]) {
        st = mpo_from_dense(ctx, terms[t].fac[m], sys->R[m], 1e-32, 0, part);
        if (!st && !key.empty()) {
          // keep a copy: the same built-in factor on the same R gives the same MPO
          Mpo* c = new Mpo();
          st = mpo_copy(ctx, part, *c);
          if (st)
            delete c;
          else
            ctx->factor_mpo_cache[key] = c;
        }
      } else {
        st = make_identity_mpo(ctx, sys->R[m], part);
      }
      if (st) {
        mpo_clear(ctx, term);
        mpo_clear(ctx, part);
        return st;
      }
      mpo_concat(term, part);
    }
    if ((st = mpo_scale(ctx, term, terms[t].coeff))) return st;
    if (out.L == 0) {
      out.L = term.L;
      out.D = term.D;
      out.core = term.core;
      term.core.clear();
    } else {
      Mpo sum;
      std::vector<const Mpo*> parts = {&out, &term};
      if ((st = mpo_stack(ctx, parts, {0, 0}, 1, sum))) return st;
      mpo_clear(ctx, out);
      mpo_clear(ctx, term);
      out.L = sum.L;
      out.D = sum.D;
      out.core = sum.core;
      sum.core.clear();
      if ((st = mpo_compress(ctx, out, tol, cap))) return st;
    }
  }
  if (terms.size() == 1 && (st = mpo_compress(ctx, out, tol, cap))) return st;
  return QLB_OK;
}

}  // namespace qlb
