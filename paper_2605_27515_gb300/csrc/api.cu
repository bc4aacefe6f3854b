// C-ABI of libqlb (declared in include/qlb.h).  Argument checking, handle
// lifetimes, operator assembly and the observables; the numerical work is in
// builder.cu, step.cu and kernels_linalg.cu.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "step.cuh"

namespace qlb {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
const char* get_error() { return g_err.c_str(); }

namespace {

inline unsigned nblk(long n, int t = 256) { return (unsigned)std::max<long>(1, (n + t - 1) / t); }

// Projector |psi><psi| as an MPO from the MPS of psi: core
// W[(t,tb)][(2s'+s)][(t',tb')] = P[t,s',t'] conj(P[tb,s,tb']).
__global__ void k_projector_core(const zd* P, int Dl, int Dr, zd* W) {
  long n = (long)Dl * Dl * 4 * Dr * Dr;
  long x = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (x >= n) return;
  long a = x / (4L * Dr * Dr);
  long rem = x % (4L * Dr * Dr);
  int p = (int)(rem / ((long)Dr * Dr));
  long b = rem % ((long)Dr * Dr);
  int t = (int)(a / Dl), tb = (int)(a % Dl);
  int t2 = (int)(b / Dr), tb2 = (int)(b % Dr);
  int so = p >> 1, si = p & 1;
  zd u = P[((long)t * 2 + so) * Dr + t2];
  zd v = P[((long)tb * 2 + si) * Dr + tb2];
  W[x] = cmul(u, cconj(v));
}

// quantics order [(s'_1 s_1) ... (s'_R s_R)] -> dense row-major
__global__ void k_tt_to_dense(const zd* T, int R, zd* O) {
  long N = 1L << R;
  long x = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (x >= N * N) return;
  long row = x / N, col = x % N;
  long idx = 0;
  for (int i = 0; i < R; i++) {
    int so = (row >> (R - 1 - i)) & 1, si = (col >> (R - 1 - i)) & 1;
    idx = idx * 4 + 2 * so + si;
  }
  O[x] = T[idx];
}

__global__ void k_normalize_vec(zd* v, long n) {
  __shared__ double sh[32];
  __shared__ double s_norm;
  double acc = 0;
  for (long x = threadIdx.x; x < n; x += blockDim.x) acc += cabs2(v[x]);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) r += sh[w];
    s_norm = r > 0 ? 1.0 / sqrt(r) : 0.0;
  }
  __syncthreads();
  for (long x = threadIdx.x; x < n; x += blockDim.x) v[x] = cscale(v[x], s_norm);
}

__global__ void k_sum_abs2_n(const zd* p, long n, double* out) {
  __shared__ double sh[32];
  double acc = 0;
  for (long x = threadIdx.x; x < n; x += blockDim.x) acc += cabs2(p[x]);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) r += sh[w];
    *out = r;
  }
}

}  // namespace

// Quantics MPS of each (normalised) mode vector by TT-SVD; chains joined.
static qlb_status product_mps(qlb_system* sys, const double* const* vecs, std::vector<zd*>& cores,
                              std::vector<int>& D) {
  qlb_ctx* ctx = sys->ctx;
  cores.clear();
  D.assign(1, 1);
  for (int m = 0; m < sys->M; m++) {
    long N = 1L << sys->R[m];
    if (!vecs[m]) {
      set_error("null mode vector");
      return QLB_EINVAL;
    }
    for (long j = 0; j < 2 * N; j++)
      if (!std::isfinite(vecs[m][j])) {
        set_error("non-finite entry in a mode vector");
        return QLB_ENONFINITE;
      }
    zd* v = nullptr;
    qlb_status s = dev_alloc(ctx, (void**)&v, sizeof(zd) * N);
    if (s) return s;
    QLB_CUDA_TRY(cudaMemcpyAsync(v, vecs[m], sizeof(zd) * N, cudaMemcpyHostToDevice, ctx->stream));
    k_normalize_vec<<<1, 256, 0, ctx->stream>>>(v, N);
    std::vector<zd*> c;
    std::vector<int> d;
    if ((s = tt_svd(ctx, v, sys->R[m], 2, 1e-30, 0, c, d))) return s;
    for (auto p : c) cores.push_back(p);
    for (int i = 1; i <= sys->R[m]; i++) D.push_back(d[i]);
  }
  return QLB_OK;
}

}  // namespace qlb

using namespace qlb;

qlb_op::~qlb_op() {
  for (auto p : owned) dev_free(nullptr, p);
  for (auto p : step_core) dev_free(nullptr, p);
}

qlb_state::~qlb_state() {
  if (stream) cudaStreamSynchronize(stream);
  if (graph) cudaGraphExecDestroy(graph);
  for (auto p : site) dev_free(nullptr, p);
  for (auto p : {X, Mb, G, Cin, Cout, T1, T2, T3, eigw, oE0, oE1, oY, oZ, Wsk}) dev_free(nullptr, p);
  dev_free(nullptr, d_lam);
  dev_free(nullptr, d_gate);
  dev_free(nullptr, d_stats);
  dev_free(nullptr, d_err);
  dev_free(nullptr, d_step);
  dev_free(nullptr, d_dims);
  if (stream) cudaStreamDestroy(stream);
}

#define QLB_API extern "C" __attribute__((visibility("default")))

#define CHECK_ARG(cond, msg)  \
  do {                        \
    if (!(cond)) {            \
      set_error(msg);         \
      return QLB_EINVAL;      \
    }                         \
  } while (0)

QLB_API void qlb_default_options(qlb_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->device = 0;
  o->precision = QLB_PREC_F64;
  o->tol = 1e-12;
  o->chi_max = 64;
  o->chi_mu_max = 16;
  o->zip_tol_factor = 1e-6;
  o->degeneracy_gap = 1e-10;
  o->max_sweeps = 40;
  o->hbm_budget = 0;
  o->stream_ordered = 0;
  o->zip_solver = 1;
  o->zip_chi_max = 0;
  o->mixed_gemm = 1;
}

QLB_API const char* qlb_last_error(void) { return get_error(); }

QLB_API qlb_status qlb_create(const qlb_options* opt, qlb_ctx** out) {
  CHECK_ARG(out, "out is null");
  *out = nullptr;
  qlb_options o;
  if (opt)
    o = *opt;
  else
    qlb_default_options(&o);
  CHECK_ARG(o.precision == QLB_PREC_F64 || o.precision == QLB_PREC_MIXED || o.precision == QLB_PREC_TC,
            "unknown precision");
  CHECK_ARG(o.tol >= 0 && o.tol < 1, "tol must be in [0, 1)");
  CHECK_ARG(o.chi_max >= 1 && o.chi_max <= 256, "chi_max must be in [1, 256]");
  CHECK_ARG(o.chi_mu_max >= 1 && o.chi_mu_max <= 128, "chi_mu_max must be in [1, 128]");
  CHECK_ARG(o.max_sweeps >= 1, "max_sweeps must be >= 1");
  CHECK_ARG(o.zip_solver == 0 || o.zip_solver == 1, "zip_solver must be 0 or 1");
  CHECK_ARG(o.mixed_gemm >= 0 && o.mixed_gemm <= 2, "mixed_gemm must be 0, 1 or 2");
  CHECK_ARG(o.zip_chi_max == 0 || (o.zip_chi_max >= o.chi_max && o.zip_chi_max <= 256),
            "zip_chi_max must be 0 or in [chi_max, 256]");
  if (o.zip_tol_factor <= 0) o.zip_tol_factor = 1e-6;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    set_error("no CUDA device available");
    return QLB_EDEVICE;
  }
  CHECK_ARG(o.device >= 0 && o.device < ndev, "device ordinal out of range");
  QLB_CUDA_TRY(cudaSetDevice(o.device));
  qlb_ctx* c = new qlb_ctx();
  c->opt = o;
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete c;
    set_error(std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    return QLB_EDEVICE;
  }
  init_kernel_attributes();
  init_qr_attributes();
  init_tc_attributes();
  {
    qlb_status st = dev_alloc(c, (void**)&c->d_solver, sizeof(double) * 16);
    if (st == QLB_OK && cudaMemset(c->d_solver, 0, sizeof(double) * 16) != cudaSuccess) st = QLB_EDEVICE;
    if (st) {
      cudaStreamDestroy(c->stream);
      delete c;
      return st;
    }
  }
  // keep freed blocks in the device pool for reuse instead of returning them to
  // the driver between allocations (process-local allocator setting)
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, o.device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  *out = c;
  return QLB_OK;
}

QLB_API void qlb_destroy(qlb_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  dev_free(ctx, ctx->d_prof);
  dev_free(ctx, ctx->d_solver);
  cudaStreamDestroy(ctx->stream);
  // buffers still held by systems, ops or states of this context no longer
  // report to it when they are freed later
  for (auto& kv : g_alloc_sizes())
    if (kv.second.second == ctx) kv.second.second = nullptr;
  delete ctx;
}

QLB_API qlb_status qlb_ctx_stream(qlb_ctx* ctx, void** stream) {
  CHECK_ARG(ctx && stream, "null argument");
  *stream = (void*)ctx->stream;
  return QLB_OK;
}

QLB_API qlb_status qlb_state_stream(qlb_state* st, void** stream) {
  CHECK_ARG(st && stream, "null argument");
  *stream = (void*)st->stream;
  return QLB_OK;
}

QLB_API qlb_status qlb_state_poll(qlb_state* st) {
  CHECK_ARG(st, "null state");
  cudaError_t e = cudaStreamQuery(st->stream);
  if (e == cudaSuccess) return QLB_OK;
  if (e == cudaErrorNotReady) {
    cudaGetLastError();
    return QLB_BUSY;
  }
  set_error(std::string("cudaStreamQuery: ") + cudaGetErrorString(e));
  return QLB_EDEVICE;
}

QLB_API qlb_status qlb_synchronize(qlb_ctx* ctx) {
  CHECK_ARG(ctx, "null context");
  QLB_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  QLB_CUDA_TRY(cudaDeviceSynchronize());
  return QLB_OK;
}

QLB_API qlb_status qlb_ctx_memory(qlb_ctx* ctx, size_t* bytes) {
  CHECK_ARG(ctx && bytes, "null argument");
  *bytes = ctx->mem_held;
  return QLB_OK;
}

QLB_API qlb_status qlb_ctx_alloc_count(qlb_ctx* ctx, int64_t* n) {
  CHECK_ARG(ctx && n, "null argument");
  *n = ctx->n_allocs;
  return QLB_OK;
}

// ------------------------------------------------------------------ systems

QLB_API qlb_status qlb_system_create(qlb_ctx* ctx, int n_modes, const int* R, qlb_system** out) {
  CHECK_ARG(ctx && R && out, "null argument");
  *out = nullptr;
  CHECK_ARG(n_modes >= 1 && n_modes <= 16, "n_modes must be in [1, 16]");
  int L = 0;
  for (int m = 0; m < n_modes; m++) {
    CHECK_ARG(R[m] >= 1 && R[m] <= 12, "R[m] must be in [1, 12]");
    L += R[m];
  }
  CHECK_ARG(L <= 64, "sum of R[m] must be <= 64");
  qlb_system* s = new qlb_system();
  s->ctx = ctx;
  s->M = n_modes;
  s->R.assign(R, R + n_modes);
  s->L = L;
  *out = s;
  return QLB_OK;
}

qlb_system::~qlb_system() { delete kraus_tmpl; }

qlb_ctx::~qlb_ctx() {
  for (auto& kv : factor_mpo_cache) delete kv.second;
}

QLB_API void qlb_system_destroy(qlb_system* sys) {
  if (!sys) return;
  dev_free(sys->ctx, sys->d_f);
  delete sys;
}

// ------------------------------------------------------------------ operators

QLB_API qlb_status qlb_op_build(qlb_system* sys, const qlb_term* terms, int n_terms, double tol, int chi_max,
                                qlb_op** out) {
  CHECK_ARG(sys && out, "null argument");
  *out = nullptr;
  CHECK_ARG(n_terms >= 1 && terms, "at least one term is needed");
  qlb_ctx* ctx = sys->ctx;
  qlb_op* op = new qlb_op();
  op->sys = sys;
  qlb_status s = QLB_OK;
  double bound = 0;
  for (int t = 0; t < n_terms && !s; t++) {
    const qlb_term& T = terms[t];
    if (!std::isfinite(T.re) || !std::isfinite(T.im)) {
      set_error("non-finite term coefficient");
      s = QLB_EINVAL;
      break;
    }
    if (T.n_factors < 0 || (T.n_factors > 0 && !T.factors)) {
      set_error("bad factor list");
      s = QLB_EINVAL;
      break;
    }
    DevTerm dt;
    dt.coeff = mk<double>(T.re, T.im);
    dt.fac.assign(sys->M, nullptr);
    dt.key.assign(sys->M, "");
    std::vector<bool> keyed(sys->M, true);
    double tb = std::sqrt(T.re * T.re + T.im * T.im);
    for (int f = 0; f < T.n_factors && !s; f++) {
      const qlb_factor& F = T.factors[f];
      if (F.mode < 0 || F.mode >= sys->M) {
        set_error("factor mode out of range");
        s = QLB_EINVAL;
        break;
      }
      int N = 1 << sys->R[F.mode];
      if (F.kind == QLB_F_DENSE && F.dense) {
        for (long j = 0; j < 2L * N * N; j++)
          if (!std::isfinite(F.dense[j])) {
            set_error("non-finite entry in a dense factor");
            s = QLB_EINVAL;
            break;
          }
        if (s) break;
      }
      int p = F.power < 1 ? 1 : F.power;
      zd* base = nullptr;
      if ((s = make_factor(ctx, N, F, &base))) break;
      op->owned.push_back(base);
      zd* acc = base;
      for (int k = 1; k < p && !s; k++) {
        zd* nx = nullptr;
        if ((s = dense_mul(ctx, acc, OP_N, base, N, &nx))) break;
        op->owned.push_back(nx);
        acc = nx;
      }
      if (s) break;
      if (dt.fac[F.mode]) {
        zd* nx = nullptr;
        if ((s = dense_mul(ctx, dt.fac[F.mode], OP_N, acc, N, &nx))) break;
        op->owned.push_back(nx);
        acc = nx;
      }
      dt.fac[F.mode] = acc;
      if (F.kind == QLB_F_DENSE) {
        keyed[F.mode] = false;
      } else {
        char piece[96];
        snprintf(piece, sizeof(piece), "%s%d^%d@%.17g", dt.key[F.mode].empty() ? "" : "*", F.kind, p,
                 F.kind == QLB_F_CHARGE ? F.param : 0.0);
        dt.key[F.mode] += piece;
      }
    }
    if (s) break;
    for (int m = 0; m < sys->M; m++)
      if (!keyed[m]) dt.key[m] = "";
    for (int m = 0; m < sys->M; m++)
      if (dt.fac[m]) tb *= dense_inf_norm(ctx, dt.fac[m], 1 << sys->R[m]);
    bound += tb;
    op->terms.push_back(dt);
  }
  if (!s) s = mpo_from_terms(sys, op->terms, tol > 0 ? tol : 1e-30, chi_max > 0 ? chi_max : 0, op->mpo);
  if (s) {
    mpo_clear(ctx, op->mpo);
    delete op;
    return s;
  }
  op->inf_norm_bound = bound;
  *out = op;
  return QLB_OK;
}

QLB_API void qlb_op_destroy(qlb_op* op) {
  if (!op) return;
  mpo_clear(op->sys->ctx, op->mpo);
  delete op;
}

QLB_API qlb_status qlb_op_bond_dims(const qlb_op* op, int* out, int cap, int* n_out) {
  CHECK_ARG(op && n_out, "null argument");
  int L = op->mpo.L;
  *n_out = L - 1;
  if (out)
    for (int i = 1; i < L && i - 1 < cap; i++) out[i - 1] = op->mpo.D[i];
  return QLB_OK;
}

static qlb_status mpo_to_dense(qlb_ctx* ctx, const Mpo& W, double* out, size_t n_doubles) {
  int L = W.L;
  CHECK_ARG(L <= 11, "dense export is for 2^L <= 2048");
  long N = 1L << L;
  CHECK_ARG(n_doubles >= (size_t)(2 * N * N), "output buffer too small");
  // T (4^i x D_i) <- T * core_i (D_i x 4 D_{i+1})
  zd* T = nullptr;
  qlb_status s;
  if ((s = dev_alloc(ctx, (void**)&T, sizeof(zd) * 4 * W.D[1]))) return s;
  QLB_CUDA_TRY(cudaMemcpyAsync(T, W.core[0], sizeof(zd) * 4 * W.D[1], cudaMemcpyDeviceToDevice, ctx->stream));
  long rows = 4;
  for (int i = 1; i < L; i++) {
    zd* nT = nullptr;
    long nn = 4L * W.D[i + 1];
    if ((s = dev_alloc(ctx, (void**)&nT, sizeof(zd) * rows * nn))) {
      dev_free(ctx, T);
      return s;
    }
    GemmDesc g{};
    g.A = T;
    g.B = W.core[i];
    g.C = nT;
    g.m = dconst((int)rows);
    g.n = dconst((int)nn);
    g.k = dconst(W.D[i]);
    g.lda = dconst(W.D[i]);
    g.ldb = dconst((int)nn);
    g.ldc = dconst((int)nn);
    g.sA1 = g.sB1 = g.sC1 = g.sA2 = g.sB2 = g.sC2 = dconst(0);
    g.nb1 = g.nb2 = dconst(1);
    g.alpha_re = 1;
    g.m_max = (int)rows;
    g.n_max = (int)nn;
    g.nb_max = 1;
    QLB_CUDA_TRY(launch_gemm<double>(g, nullptr, ctx->stream, nullptr));
    dev_free(ctx, T);
    T = nT;
    rows *= 4;
  }
  zd* O = nullptr;
  if ((s = dev_alloc(ctx, (void**)&O, sizeof(zd) * N * N))) {
    dev_free(ctx, T);
    return s;
  }
  k_tt_to_dense<<<nblk(N * N), 256, 0, ctx->stream>>>(T, L, O);
  QLB_CUDA_TRY(cudaMemcpyAsync(out, O, sizeof(zd) * N * N, cudaMemcpyDeviceToHost, ctx->stream));
  QLB_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  dev_free(ctx, T);
  dev_free(ctx, O);
  return QLB_OK;
}

QLB_API qlb_status qlb_op_to_dense(const qlb_op* op, double* out, size_t n_doubles) {
  CHECK_ARG(op && out, "null argument");
  return mpo_to_dense(op->sys->ctx, op->mpo, out, n_doubles);
}

QLB_API qlb_status qlb_kraus_to_dense(qlb_state* st, double dt, int k, double* out, size_t n_doubles) {
  CHECK_ARG(st && out, "null argument");
  CHECK_ARG(std::isfinite(dt) && dt > 0, "dt must be positive and finite");
  qlb_status s;
  bool rebuilt = !(st->kraus.dt == dt && st->kraus.version == st->sys->version);
  if ((s = build_kraus(st, dt))) return s;
  if (rebuilt && (s = plan_buffers(st, st->kraus))) return s;
  Mpo W;
  if ((s = kraus_branch(st, k, W))) {
    mpo_clear(st->sys->ctx, W);
    return s;
  }
  s = mpo_to_dense(st->sys->ctx, W, out, n_doubles);
  mpo_clear(st->sys->ctx, W);
  return s;
}

QLB_API qlb_status qlb_state_to_dense(qlb_state* st, double* out, size_t n_doubles, int* chi_mu_out) {
  CHECK_ARG(st && out && chi_mu_out, "null argument");
  CHECK_ARG(st->L <= 12, "dense export is for 2^L <= 4096");
  qlb_ctx* ctx = st->sys->ctx;
  std::vector<int> d;
  qlb_status s;
  if ((s = read_dims(st, d))) return s;
  const int L = st->L;
  const long N = 1L << L;
  const int mu = d[0];
  *chi_mu_out = mu;
  CHECK_ARG(n_doubles >= (size_t)(2 * N * mu), "output buffer too small");
  // T[(mu, s_0..s_i), r_{i+1}] = T[(mu, s_0..s_{i-1}), r_i] * A_i[r_i][(s_i, r_{i+1})]
  zd* T = nullptr;
  long rows = mu;
  if ((s = dev_alloc(ctx, (void**)&T, sizeof(zd) * mu * 2 * d[1]))) return s;
  QLB_CUDA_TRY(cudaMemcpyAsync(T, st->site[0], sizeof(zd) * mu * 2 * d[1], cudaMemcpyDeviceToDevice, st->stream));
  rows *= 2;
  for (int i = 1; i < L; i++) {
    zd* nT = nullptr;
    long nn = 2L * d[i + 1];
    if ((s = dev_alloc(ctx, (void**)&nT, sizeof(zd) * rows * nn))) {
      dev_free(ctx, T);
      return s;
    }
    GemmDesc g{};
    g.A = T;
    g.B = st->site[i];
    g.C = nT;
    g.m = dconst((int)rows);
    g.n = dconst((int)nn);
    g.k = dconst(d[i]);
    g.lda = dconst(d[i]);
    g.ldb = dconst((int)nn);
    g.ldc = dconst((int)nn);
    g.sA1 = g.sB1 = g.sC1 = g.sA2 = g.sB2 = g.sC2 = dconst(0);
    g.nb1 = g.nb2 = dconst(1);
    g.alpha_re = 1;
    g.m_max = (int)rows;
    g.n_max = (int)nn;
    g.nb_max = 1;
    QLB_CUDA_TRY(launch_gemm<double>(g, nullptr, st->stream, nullptr));
    dev_free(ctx, T);
    T = nT;
    rows *= 2;
  }
  std::vector<zd> h((size_t)mu * N);
  QLB_CUDA_TRY(cudaMemcpyAsync(h.data(), T, sizeof(zd) * h.size(), cudaMemcpyDeviceToHost, st->stream));
  QLB_CUDA_TRY(cudaStreamSynchronize(st->stream));
  dev_free(ctx, T);
  // h is [(mu, n)] ; out is [n][mu]
  for (int m = 0; m < mu; m++)
    for (long n = 0; n < N; n++) {
      out[2 * (n * mu + m)] = h[(size_t)m * N + n].re;
      out[2 * (n * mu + m) + 1] = h[(size_t)m * N + n].im;
    }
  return QLB_OK;
}

QLB_API qlb_status qlb_set_hamiltonian(qlb_system* sys, const qlb_op* H0, const qlb_op* H1, const double* f_table,
                                       int64_t n_f) {
  CHECK_ARG(sys, "null system");
  CHECK_ARG(!H0 || H0->sys == sys, "H0 belongs to another system");
  CHECK_ARG(!H1 || H1->sys == sys, "H1 belongs to another system");
  CHECK_ARG(!H1 || (f_table && n_f > 0), "H1 needs a drive table");
  sys->H0 = H0;
  sys->H1 = H1;
  dev_free(sys->ctx, sys->d_f);
  sys->d_f = nullptr;
  sys->n_f = 0;
  if (H1) {
    for (int64_t j = 0; j < n_f; j++)
      CHECK_ARG(std::isfinite(f_table[j]), "non-finite drive table entry");
    qlb_status s = dev_alloc(sys->ctx, (void**)&sys->d_f, sizeof(double) * n_f);
    if (s) return s;
    QLB_CUDA_TRY(cudaMemcpy(sys->d_f, f_table, sizeof(double) * n_f, cudaMemcpyHostToDevice));
    sys->n_f = n_f;
  }
  sys->version++;
  return QLB_OK;
}

QLB_API qlb_status qlb_add_jump(qlb_system* sys, const qlb_op* L) {
  CHECK_ARG(sys && L, "null argument");
  CHECK_ARG(L->sys == sys, "jump operator belongs to another system");
  CHECK_ARG(sys->jumps.size() < 15, "at most 15 jump operators");
  sys->jumps.push_back(L);
  sys->version++;
  return QLB_OK;
}

QLB_API qlb_status qlb_set_scheme(qlb_system* sys, int order) {
  CHECK_ARG(sys, "null argument");
  CHECK_ARG(order == 1 || order == 2, "scheme order must be 1 or 2");
  CHECK_ARG(order == 1 || !sys->H1, "the second-order scheme needs a time-independent Hamiltonian");
  CHECK_ARG(order == 1 || sys->jumps.size() <= 6, "the second-order scheme takes at most 6 jump operators");
  if (sys->order != order) {
    sys->order = order;
    sys->version++;
  }
  return QLB_OK;
}

// ------------------------------------------------------------------ states

QLB_API qlb_status qlb_state_init_product(qlb_system* sys, const double* const* mode_vecs, qlb_state** out) {
  CHECK_ARG(sys && mode_vecs && out, "null argument");
  *out = nullptr;
  qlb_ctx* ctx = sys->ctx;
  qlb_state* st = new qlb_state();
  st->sys = sys;
  st->L = sys->L;
  st->prec = ctx->opt.precision;
  st->tol = ctx->opt.tol;
  st->chi_max = st->cap_chi = ctx->opt.chi_max;
  st->chi_mu_max = st->cap_mu = ctx->opt.chi_mu_max;
  const int L = st->L;
  qlb_status s;
  std::vector<zd*> cores;
  std::vector<int> D;
  auto fail = [&](qlb_status code) {
    for (auto p : cores) dev_free(ctx, p);
    delete st;
    return code;
  };
  if ((s = product_mps(sys, mode_vecs, cores, D))) return fail(s);
  if ((s = dev_alloc(ctx, (void**)&st->d_dims, sizeof(int) * (2 * L + 8)))) return fail(s);
  if ((s = dev_alloc(ctx, (void**)&st->d_stats, sizeof(double) * 8))) return fail(s);
  if ((s = dev_alloc(ctx, (void**)&st->d_err, sizeof(int) * 4))) return fail(s);
  if ((s = dev_alloc(ctx, (void**)&st->d_step, sizeof(long long)))) return fail(s);
  std::vector<int> hd(2 * L + 8, 1);
  for (int i = 0; i <= L; i++) hd[i] = D[i];
  for (int i = 0; i <= L; i++) hd[L + 1 + i] = D[i];
  QLB_CUDA_TRY(cudaMemcpy(st->d_dims, hd.data(), sizeof(int) * hd.size(), cudaMemcpyHostToDevice));
  if (cudaStreamCreateWithFlags(&st->stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("cudaStreamCreate failed");
    delete st;
    return QLB_EDEVICE;
  }
  QLB_CUDA_TRY(cudaMemsetAsync(st->d_stats, 0, sizeof(double) * 8, st->stream));
  QLB_CUDA_TRY(cudaMemsetAsync(st->d_err, 0, sizeof(int) * 4, st->stream));
  QLB_CUDA_TRY(cudaMemsetAsync(st->d_step, 0, sizeof(long long), st->stream));
  st->site = cores;
  cores.clear();
  st->site_cap.assign(L, 0);
  for (int i = 0; i < L; i++) st->site_cap[i] = (size_t)D[i] * 2 * D[i + 1];
  if ((s = truncate_pass(st))) {
    delete st;
    return s;
  }
  *out = st;
  return QLB_OK;
}

QLB_API void qlb_state_destroy(qlb_state* st) {
  if (!st) return;
  cudaStreamSynchronize(st->stream);
  delete st;
}

QLB_API qlb_status qlb_truncate(qlb_state* st, double tol, int chi_max, int chi_mu_max) {
  CHECK_ARG(st, "null state");
  CHECK_ARG(tol < 1, "tol must be < 1");
  CHECK_ARG(chi_max <= st->cap_chi, "chi_max above the allocation cap of this state");
  CHECK_ARG(chi_mu_max <= st->cap_mu, "chi_mu_max above the allocation cap of this state");
  if (tol > 0) st->tol = tol;
  if (chi_max > 0) st->chi_max = chi_max;
  if (chi_mu_max > 0) st->chi_mu_max = chi_mu_max;
  st->plan_key++;  // caps are baked into captured graphs
  return truncate_pass(st);
}

QLB_API qlb_status qlb_step(qlb_state* st, double dt, int64_t n) {
  CHECK_ARG(st, "null state");
  CHECK_ARG(std::isfinite(dt) && dt > 0, "dt must be positive and finite");
  CHECK_ARG(n >= 0, "n must be >= 0");
  qlb_status s;
  bool rebuilt = !(st->kraus.dt == dt && st->kraus.version == st->sys->version);
  if ((s = build_kraus(st, dt))) return s;
  if (rebuilt && (s = plan_buffers(st, st->kraus))) return s;
  if ((s = run_steps(st, n, !st->sys->ctx->opt.stream_ordered))) return s;
  return st->kraus.unstable_factor > 4.0 ? QLB_WUNSTABLE : QLB_OK;
}

QLB_API qlb_status qlb_expectation(qlb_state* st, const qlb_op* O, double* out) {
  CHECK_ARG(st && O && out, "null argument");
  CHECK_ARG(O->sys == st->sys, "operator belongs to another system");
  qlb_op* op = const_cast<qlb_op*>(O);
  if (op->step_core.empty()) {
    qlb_ctx* ctx = st->sys->ctx;
    std::vector<zd*> c;
    qlb_status s = mpo_step_layout(ctx, op->mpo, c, ctx->stream);
    if (s == QLB_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
      set_error("step-layout conversion of the operator failed");
      s = QLB_EDEVICE;
    }
    if (s) {
      for (auto p : c) dev_free(ctx, p);
      return s;
    }
    op->step_core = c;
  }
  return expectation_mpo(st, op->step_core, op->mpo.D, out);
}

QLB_API qlb_status qlb_fidelity(qlb_state* st, const double* const* target, double* out) {
  CHECK_ARG(st && target && out, "null argument");
  qlb_system* sys = st->sys;
  qlb_ctx* ctx = sys->ctx;
  std::vector<zd*> P;
  std::vector<int> D;
  qlb_status s = product_mps(sys, target, P, D);
  if (s) return s;
  Mpo W;
  W.L = st->L;
  W.D.assign(st->L + 1, 1);
  W.core.assign(st->L, nullptr);
  for (int i = 0; i <= st->L; i++) W.D[i] = D[i] * D[i];
  for (int i = 0; i < st->L && !s; i++) {
    long n = (long)W.D[i] * 4 * W.D[i + 1];
    if ((s = dev_alloc(ctx, (void**)&W.core[i], sizeof(zd) * n))) break;
    k_projector_core<<<nblk(n), 256, 0, ctx->stream>>>(P[i], D[i], D[i + 1], W.core[i]);
  }
  std::vector<zd*> Ws;
  if (!s) s = mpo_step_layout(ctx, W, Ws, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  for (auto p : P) dev_free(ctx, p);
  double r[2] = {0, 0};
  if (!s) s = expectation_mpo(st, Ws, W.D, r);
  for (auto p : Ws) dev_free(ctx, p);
  mpo_clear(ctx, W);
  if (s) return s;
  *out = r[0];
  return QLB_OK;
}

QLB_API qlb_status qlb_trace(qlb_state* st, double* out) {
  CHECK_ARG(st && out, "null argument");
  return state_sum_abs2_site0(st, out);
}

QLB_API qlb_status qlb_purity(qlb_state* st, double* out) {
  CHECK_ARG(st && out, "null argument");
  qlb_ctx* ctx = st->sys->ctx;
  std::vector<int> d;
  qlb_status s;
  if ((s = read_dims(st, d))) return s;
  int mu = d[0], r = d[1];
  zd* G = nullptr;
  double* acc = nullptr;
  if ((s = dev_alloc(ctx, (void**)&G, sizeof(zd) * mu * mu))) return s;
  if ((s = dev_alloc(ctx, (void**)&acc, sizeof(double)))) {
    dev_free(ctx, G);
    return s;
  }
  GemmDesc g{};
  g.A = st->site[0];
  g.B = st->site[0];
  g.C = G;
  g.m = g.n = dconst(mu);
  g.k = dconst(2 * r);
  g.opB = OP_C;
  g.lda = g.ldb = dconst(2 * r);
  g.ldc = dconst(mu);
  g.sA1 = g.sB1 = g.sC1 = g.sA2 = g.sB2 = g.sC2 = dconst(0);
  g.nb1 = g.nb2 = dconst(1);
  g.alpha_re = 1;
  g.m_max = g.n_max = mu;
  g.nb_max = 1;
  QLB_CUDA_TRY(launch_gemm<double>(g, nullptr, st->stream, nullptr));
  k_sum_abs2_n<<<1, 256, 0, st->stream>>>(G, (long)mu * mu, acc);
  double h = 0, tr = 0;
  QLB_CUDA_TRY(cudaMemcpyAsync(&h, acc, sizeof(double), cudaMemcpyDeviceToHost, st->stream));
  QLB_CUDA_TRY(cudaStreamSynchronize(st->stream));
  dev_free(ctx, G);
  dev_free(ctx, acc);
  if ((s = state_sum_abs2_site0(st, &tr))) return s;
  *out = tr > 0 ? h / (tr * tr) : 0.0;
  return QLB_OK;
}

QLB_API qlb_status qlb_bond_dims(qlb_state* st, int* out, int cap, int* n_out) {
  CHECK_ARG(st && n_out, "null argument");
  std::vector<int> d;
  qlb_status s = read_dims(st, d);
  if (s) return s;
  *n_out = st->L;
  if (out)
    for (int i = 0; i < st->L && i < cap; i++) out[i] = d[i];
  return QLB_OK;
}

QLB_API qlb_status qlb_step_stats(qlb_state* st, double* out4) {
  CHECK_ARG(st && out4, "null argument");
  double h[4];
  QLB_CUDA_TRY(cudaStreamSynchronize(st->stream));
  QLB_CUDA_TRY(cudaMemcpy(h, st->d_stats, sizeof(h), cudaMemcpyDeviceToHost));
  long long steps = 0;
  QLB_CUDA_TRY(cudaMemcpy(&steps, st->d_step, sizeof(steps), cudaMemcpyDeviceToHost));
  out4[0] = h[1];
  out4[1] = h[2];
  out4[2] = st->kraus.unstable_factor;
  out4[3] = (double)steps;
  return QLB_OK;
}

// ------------------------------------------------------------------ checkpoint

struct ExportHeader {
  uint64_t magic;
  int32_t L;
  int32_t pad;
};
static const uint64_t QLB_MAGIC = 0x31424c51u;  // "QLB1"

QLB_API qlb_status qlb_state_export(qlb_state* st, void* out, size_t cap, size_t* n_bytes) {
  CHECK_ARG(st && n_bytes, "null argument");
  std::vector<int> d;
  qlb_status s = read_dims(st, d);
  if (s) return s;
  const int L = st->L;
  size_t need = sizeof(ExportHeader) + sizeof(int) * (L + 1);
  for (int i = 0; i < L; i++) need += sizeof(zd) * (size_t)d[i] * 2 * d[i + 1];
  *n_bytes = need;
  if (!out) return QLB_OK;
  CHECK_ARG(cap >= need, "export buffer too small");
  char* p = (char*)out;
  ExportHeader h{QLB_MAGIC, L, 0};
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  std::memcpy(p, d.data(), sizeof(int) * (L + 1));
  p += sizeof(int) * (L + 1);
  for (int i = 0; i < L; i++) {
    size_t b = sizeof(zd) * (size_t)d[i] * 2 * d[i + 1];
    QLB_CUDA_TRY(cudaMemcpy(p, st->site[i], b, cudaMemcpyDeviceToHost));
    p += b;
  }
  return QLB_OK;
}

QLB_API qlb_status qlb_state_import(qlb_state* st, const void* in, size_t n_bytes) {
  CHECK_ARG(st && in, "null argument");
  const int L = st->L;
  CHECK_ARG(n_bytes >= sizeof(ExportHeader) + sizeof(int) * (L + 1), "import buffer too small");
  const char* p = (const char*)in;
  ExportHeader h;
  std::memcpy(&h, p, sizeof(h));
  CHECK_ARG(h.magic == QLB_MAGIC && h.L == L, "import buffer is not a state of this system");
  p += sizeof(h);
  std::vector<int> d(L + 1);
  std::memcpy(d.data(), p, sizeof(int) * (L + 1));
  p += sizeof(int) * (L + 1);
  size_t need = sizeof(ExportHeader) + sizeof(int) * (L + 1);
  CHECK_ARG(d[0] >= 1 && d[0] <= st->cap_mu && d[L] == 1, "bad purification rank in import");
  for (int i = 1; i < L; i++) CHECK_ARG(d[i] >= 1 && d[i] <= st->cap_chi, "bond above the state's cap");
  for (int i = 0; i < L; i++) need += sizeof(zd) * (size_t)d[i] * 2 * d[i + 1];
  CHECK_ARG(n_bytes >= need, "import buffer too small");
  qlb_ctx* ctx = st->sys->ctx;
  for (int i = 0; i < L; i++) {
    size_t ne = (size_t)d[i] * 2 * d[i + 1];
    if (ne > st->site_cap[i]) {
      zd* q = nullptr;
      qlb_status s = dev_alloc(ctx, (void**)&q, sizeof(zd) * ne);
      if (s) return s;
      dev_free(ctx, st->site[i]);
      st->site[i] = q;
      st->site_cap[i] = ne;
      st->plan_key++;
    }
    QLB_CUDA_TRY(cudaMemcpy(st->site[i], p, sizeof(zd) * ne, cudaMemcpyHostToDevice));
    p += sizeof(zd) * ne;
  }
  std::vector<int> hd(2 * L + 8, 1);
  for (int i = 0; i <= L; i++) hd[i] = hd[L + 1 + i] = d[i];
  QLB_CUDA_TRY(cudaMemcpy(st->d_dims, hd.data(), sizeof(int) * (2 * L + 2), cudaMemcpyHostToDevice));
  return QLB_OK;
}

// ------------------------------------------------------------------ profiling

QLB_API qlb_status qlb_profile_enable(qlb_ctx* ctx, int on) {
  CHECK_ARG(ctx, "null context");
  if (on && !ctx->d_prof) {
    qlb_status s = dev_alloc(ctx, (void**)&ctx->d_prof, sizeof(double) * 2 * QLB_K_COUNT);
    if (s) return s;
    QLB_CUDA_TRY(cudaMemset(ctx->d_prof, 0, sizeof(double) * 2 * QLB_K_COUNT));
  }
  ctx->prof_on = on != 0;
  return QLB_OK;
}

static qlb_status prof_collect(qlb_ctx* ctx) {
  QLB_CUDA_TRY(cudaDeviceSynchronize());
  for (auto& e : ctx->prof_events) {
    float ms = 0;
    QLB_CUDA_TRY(cudaEventElapsedTime(&ms, e.a, e.b));
    ctx->prof_ms[e.kclass] += ms;
    ctx->prof_launch[e.kclass] += 1;
  }
  ctx->prof_events.clear();
  ctx->ev_used = 0;
  return QLB_OK;
}

QLB_API qlb_status qlb_profile_read(qlb_ctx* ctx, int kclass, double* ms, int64_t* launches, double* flops,
                                    double* bytes) {
  CHECK_ARG(ctx, "null context");
  CHECK_ARG(kclass >= 0 && kclass < QLB_K_COUNT, "bad kernel class");
  qlb_status s = prof_collect(ctx);
  if (s) return s;
  double h[2 * QLB_K_COUNT] = {0};
  if (ctx->d_prof) QLB_CUDA_TRY(cudaMemcpy(h, ctx->d_prof, sizeof(h), cudaMemcpyDeviceToHost));
  if (ms) *ms = ctx->prof_ms[kclass];
  if (launches) *launches = ctx->prof_launch[kclass];
  if (flops) *flops = h[kclass];
  if (bytes) *bytes = h[QLB_K_COUNT + kclass];
  return QLB_OK;
}

QLB_API qlb_status qlb_profile_reset(qlb_ctx* ctx) {
  CHECK_ARG(ctx, "null context");
  qlb_status s = prof_collect(ctx);
  if (s) return s;
  for (int k = 0; k < QLB_K_COUNT; k++) {
    ctx->prof_ms[k] = 0;
    ctx->prof_launch[k] = 0;
  }
  if (ctx->d_prof) QLB_CUDA_TRY(cudaMemset(ctx->d_prof, 0, sizeof(double) * 2 * QLB_K_COUNT));
  QLB_CUDA_TRY(cudaDeviceSynchronize());
  if (ctx->d_solver) QLB_CUDA_TRY(cudaMemset(ctx->d_solver, 0, sizeof(double) * 16));
  return QLB_OK;
}

QLB_API qlb_status qlb_profile_solver_stats(qlb_ctx* ctx, double* out, int n_out) {
  CHECK_ARG(ctx && out && n_out >= 0, "null argument");
  QLB_CUDA_TRY(cudaDeviceSynchronize());
  double h[16] = {0};
  if (ctx->d_solver) QLB_CUDA_TRY(cudaMemcpy(h, ctx->d_solver, sizeof(h), cudaMemcpyDeviceToHost));
  for (int i = 0; i < n_out && i < 9; i++) out[i] = h[i];
  return QLB_OK;
}

// ------------------------------------------------------------------ tensor-core GEMM check

QLB_API qlb_status qlb_tc_zgemm(int device, int m, int n, int k, const double* A, const double* B, double* C) {
  CHECK_ARG(A && B && C, "null argument");
  CHECK_ARG(m >= 1 && n >= 1 && k >= 0 && (long)m * n <= (1L << 26) && (long)m * k <= (1L << 26) &&
                (long)k * n <= (1L << 26),
            "sizes out of range");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    set_error("qlb_tc_zgemm: no such CUDA device");
    return QLB_EDEVICE;
  }
  QLB_CUDA_TRY(cudaSetDevice(device));
  init_tc_attributes();
  zd *dA = nullptr, *dB = nullptr, *dC = nullptr;
  int* derr = nullptr;
  auto cleanup = [&]() {
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(derr);
  };
  if (cudaMalloc(&dA, sizeof(zd) * std::max<long>(1, (long)m * k)) != cudaSuccess ||
      cudaMalloc(&dB, sizeof(zd) * std::max<long>(1, (long)k * n)) != cudaSuccess ||
      cudaMalloc(&dC, sizeof(zd) * (long)m * n) != cudaSuccess || cudaMalloc(&derr, sizeof(int)) != cudaSuccess) {
    cleanup();
    set_error("qlb_tc_zgemm: device allocation failed");
    return QLB_ENOMEM;
  }
  cudaMemcpy(dA, A, sizeof(zd) * (long)m * k, cudaMemcpyHostToDevice);
  cudaMemcpy(dB, B, sizeof(zd) * (long)k * n, cudaMemcpyHostToDevice);
  cudaMemset(derr, 0, sizeof(int));
  GemmDesc g{};
  g.A = dA;
  g.B = dB;
  g.C = dC;
  g.m = dconst(m);
  g.n = dconst(n);
  g.k = dconst(k);
  g.lda = dconst(k);
  g.ldb = dconst(n);
  g.ldc = dconst(n);
  g.sA1 = g.sB1 = g.sC1 = g.sA2 = g.sB2 = g.sC2 = dconst(0);
  g.nb1 = g.nb2 = dconst(1);
  g.alpha_re = 1.0;
  g.m_max = m;
  g.n_max = n;
  g.nb_max = 1;
  cudaError_t e = launch_gemm_tc(g, nullptr, 0, derr, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(C, dC, sizeof(zd) * (long)m * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
  cleanup();
  if (e != cudaSuccess) {
    set_error(std::string("qlb_tc_zgemm: ") + cudaGetErrorString(e));
    return QLB_EDEVICE;
  }
  if (herr) {
    set_error("qlb_tc_zgemm: a bounded wait for the tensor-core pipeline gave up");
    return QLB_ETIMEOUT;
  }
  return QLB_OK;
}

// ------------------------------------------------------------------ truncation-solver check

QLB_API qlb_status qlb_eig_check(int device, int precision, int solver, int n, const double* G, double tol, int cap,
                                 double* lam, double* V, int* k_out, double* ms) {
  CHECK_ARG(G && lam && V && k_out && ms, "null argument");
  CHECK_ARG(n >= 1 && n <= 512, "n must be in [1, 512]");
  CHECK_ARG(precision == QLB_PREC_F64 || precision == QLB_PREC_MIXED, "precision must be F64 or MIXED");
  CHECK_ARG(solver >= 0 && solver <= 5, "unknown solver");
  CHECK_ARG(tol >= 0 && tol < 1 && cap >= 1, "bad truncation parameters");
  CHECK_ARG(solver != 2 || n <= 128, "the 8-CTA cluster solve takes n <= 128");
  CHECK_ARG(solver != 3 || n <= 256, "the 16-CTA cluster solve takes n <= 256");
  CHECK_ARG(solver != 4 || (precision == QLB_PREC_F64 && n <= 64), "the QL solve is FP64 with n <= 64");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    set_error("qlb_eig_check: no such CUDA device");
    return QLB_EDEVICE;
  }
  QLB_CUDA_TRY(cudaSetDevice(device));
  init_kernel_attributes();
  init_qr_attributes();
  for (long i = 0; i < 2L * n * n; i++)
    if (!std::isfinite(G[i])) {
      set_error("qlb_eig_check: non-finite input");
      return QLB_ENONFINITE;
    }
  const size_t nn = (size_t)n * n;
  size_t ws = std::max(eig_workspace_elems(n), zipqr_workspace_elems(n));
  ws = std::max(ws, 2 * (size_t)(n + 1) * (n + 1));  // G and V of the padded size in a global workspace
  zd *dG = nullptr, *dG0 = nullptr, *dOut = nullptr, *dW = nullptr;
  double* dLam = nullptr;
  int *dDims = nullptr, *dErr = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    cudaFree(dG);
    cudaFree(dG0);
    cudaFree(dOut);
    cudaFree(dW);
    cudaFree(dLam);
    cudaFree(dDims);
    cudaFree(dErr);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(&dG, sizeof(zd) * nn) != cudaSuccess || cudaMalloc(&dG0, sizeof(zd) * nn) != cudaSuccess ||
      cudaMalloc(&dOut, sizeof(zd) * nn) != cudaSuccess || cudaMalloc(&dW, sizeof(zd) * ws) != cudaSuccess ||
      cudaMalloc(&dLam, sizeof(double) * n) != cudaSuccess || cudaMalloc(&dDims, sizeof(int) * 4) != cudaSuccess ||
      cudaMalloc(&dErr, sizeof(int)) != cudaSuccess) {
    cleanup();
    set_error("qlb_eig_check: device allocation failed");
    return QLB_ENOMEM;
  }
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaMemcpy(dG0, G, sizeof(zd) * nn, cudaMemcpyHostToDevice);
  cudaMemset(dLam, 0, sizeof(double) * n);
  // dims[0] = n, dims[1] = kept count, dims[2] = gate
  EigDesc e{};
  e.G = dG;
  e.n = dconst(n);
  e.n_max = n;
  e.out = dOut;
  e.out_mode = 0;
  e.dim_out = 1;
  e.tol = tol;
  e.cap = dconst(cap);
  e.gap = 1e-10;
  e.max_sweeps = 40;
  e.err = dErr;
  if (solver != 5) e.lam = dLam;
  const bool mixed = precision == QLB_PREC_MIXED;
  cudaError_t r = cudaSuccess;
  float t = 0.f;
  for (int rep = 0; rep < 2 && r == cudaSuccess; rep++) {
    cudaMemcpy(dG, dG0, sizeof(zd) * nn, cudaMemcpyDeviceToDevice);
    cudaMemset(dDims, 0, sizeof(int) * 4);
    cudaMemset(dErr, 0, sizeof(int));
    cudaEventRecord(e0, 0);
    if (solver == 5) e.gate = dDims + 2;
    r = launch_solver(mixed, solver, e, dDims, 0, dW);
    cudaEventRecord(e1, 0);
    if (r == cudaSuccess) r = cudaEventSynchronize(e1);
    if (r == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
  }
  int hd[4] = {0, 0, 0, 0}, herr = 0;
  if (r == cudaSuccess) r = cudaMemcpy(hd, dDims, sizeof(hd), cudaMemcpyDeviceToHost);
  if (r == cudaSuccess) r = cudaMemcpy(&herr, dErr, sizeof(int), cudaMemcpyDeviceToHost);
  const bool gated = solver == 5 && hd[2] != 0;
  const int k = gated ? 0 : std::max(0, std::min(hd[1], n));
  if (r == cudaSuccess) r = cudaMemcpy(lam, dLam, sizeof(double) * n, cudaMemcpyDeviceToHost);
  if (r == cudaSuccess && k > 0) r = cudaMemcpy(V, dOut, sizeof(zd) * (size_t)n * k, cudaMemcpyDeviceToHost);
  cleanup();
  if (r != cudaSuccess) {
    set_error(std::string("qlb_eig_check: ") + cudaGetErrorString(r));
    return QLB_EDEVICE;
  }
  *k_out = gated ? -1 : k;
  *ms = t;
  if (herr & 2) {
    set_error("qlb_eig_check: non-finite values in the solve");
    return QLB_ENONFINITE;
  }
  if (herr & 1) {
    set_error("qlb_eig_check: the Jacobi solve hit its sweep limit");
    return QLB_ENOTCONV;
  }
  return QLB_OK;
}

// ------------------------------------------------------------------ GEMM engine check

QLB_API qlb_status qlb_zgemm_check(int device, int engine, int m, int n, int k, const double* A, const double* B,
                                   double* C, double* ms) {
  CHECK_ARG(A && B && C && ms, "null argument");
  CHECK_ARG(engine >= 0 && engine <= 2, "unknown engine");
  CHECK_ARG(m >= 1 && n >= 1 && k >= 0 && (long)m * n <= (1L << 26) && (long)m * k <= (1L << 26) &&
                (long)k * n <= (1L << 26),
            "sizes out of range");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    set_error("qlb_zgemm_check: no such CUDA device");
    return QLB_EDEVICE;
  }
  QLB_CUDA_TRY(cudaSetDevice(device));
  init_tc_attributes();
  const size_t nws = gemm_workspace_elems(gemm_grid_default());
  zd *dA = nullptr, *dB = nullptr, *dC = nullptr, *dW = nullptr;
  int* derr = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(dW);
    cudaFree(derr);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(&dA, sizeof(zd) * std::max<long>(1, (long)m * k)) != cudaSuccess ||
      cudaMalloc(&dB, sizeof(zd) * std::max<long>(1, (long)k * n)) != cudaSuccess ||
      cudaMalloc(&dC, sizeof(zd) * (long)m * n) != cudaSuccess || cudaMalloc(&dW, sizeof(zd) * nws) != cudaSuccess ||
      cudaMalloc(&derr, sizeof(int)) != cudaSuccess) {
    cleanup();
    set_error("qlb_zgemm_check: device allocation failed");
    return QLB_ENOMEM;
  }
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaMemcpy(dA, A, sizeof(zd) * (long)m * k, cudaMemcpyHostToDevice);
  cudaMemcpy(dB, B, sizeof(zd) * (long)k * n, cudaMemcpyHostToDevice);
  cudaMemset(dW, 0, sizeof(zd) * nws);
  cudaMemset(derr, 0, sizeof(int));
  GemmDesc g{};
  g.A = dA;
  g.B = dB;
  g.C = dC;
  g.m = dconst(m);
  g.n = dconst(n);
  g.k = dconst(k);
  g.lda = dconst(k);
  g.ldb = dconst(n);
  g.ldc = dconst(n);
  g.sA1 = g.sB1 = g.sC1 = g.sA2 = g.sB2 = g.sC2 = dconst(0);
  g.nb1 = g.nb2 = dconst(1);
  g.alpha_re = 1.0;
  g.m_max = m;
  g.n_max = n;
  g.nb_max = 1;
  g.ws = dW;
  g.df64 = engine == 1;
  cudaError_t e = cudaSuccess;
  float t = 0.f;
  for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {
    cudaEventRecord(e0, 0);
    e = engine == 2 ? launch_gemm_tc(g, nullptr, 0, derr, nullptr) : launch_gemm<double>(g, nullptr, 0, nullptr);
    cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(C, dC, sizeof(zd) * (long)m * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
  cleanup();
  if (e != cudaSuccess) {
    set_error(std::string("qlb_zgemm_check: ") + cudaGetErrorString(e));
    return QLB_EDEVICE;
  }
  *ms = t;
  if (herr) {
    set_error("qlb_zgemm_check: a bounded wait for the tensor-core pipeline gave up");
    return QLB_ETIMEOUT;
  }
  return QLB_OK;
}
