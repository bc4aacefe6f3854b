// One time step of the purified quantics MPS (Sec. V.B with Sec. V.A and IV.A):
//
//   zip-up, left to right, site i = 0..L-1 (MPO.MPS product, Sec. III.A):
//     X[l',a,(s,r)]   = sum_l  C[l',l,a] A_i[l,s,r]                   (batched GEMM over l')
//     M[(l',s'),(r,b)] = sum_{a,s} X[l',a,s,r] W_i[s',a,s,b]          (batched GEMM over l', s')
//     G = M M^dag ; eigen(G) ; keep k columns U (relative weight tol*zip_tol_factor)
//     A_i <- U ; C' = U^dag M  (carry [k][r][b] into site i+1)
//   site 0 starts from the identity carry on (mu, k): the branch index k of the
//   stacked Kraus MPO multiplies the purification index (matrix addition, Sec. V.A);
//   right to left, bond i = L-1..1 (compression after the addition, Sec. V.A):
//     G = M^dag M with M = A_i as [l] x [(s,r)] ; eigen ; keep k rows V^dag (tol, chi_max)
//     A_i <- V^dag ; A_{i-1} <- A_{i-1} (M V)
//   purification rank (Sec. IV.A): G = A_0 A_0^dag over mu ; keep the top chi_mu
//     eigenvectors Y ; A_0 <- Y^dag A_0 / sqrt(kept weight)   (rho / Tr rho, Sec. V.B).
//
// Every shape is a DimExpr over the device dims array, so the whole step is a
// fixed launch sequence (captured once as a CUDA graph) whose kernels read the
// current bond dimensions from device memory.

#include <algorithm>
#include <cmath>
#include <cstring>

#include "df64.cuh"
#include "step.cuh"

namespace qlb {

namespace {

inline unsigned nblk(long n, int t = 256) { return (unsigned)std::max<long>(1, (n + t - 1) / t); }

// z_0 = chi_mu * B, z_L = 1; identity carry C0[(mu*B + k)][mu0][k0] = delta delta;
// drive coefficient rewrite of the H1 block of core 0; reset per-step stats.
__device__ void step_begin_body(const StepBeginArgs& a) {
  int* d = a.d;
  const int L = a.L, B = a.B;
  int mu = d[0];
  int zl = mu * B;
  long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const long stride = (long)gridDim.x * blockDim.x;
  if (tid == 0) {
    d[L + 1] = zl;
    d[2 * L + 1] = 1;
    a.stats[2] = 0.0;
  }
  long n = (long)zl * mu * B;
  for (long x = tid; x < n && x < a.c0_cap; x += stride) {
    long lp = x / ((long)mu * B);
    long rem = x % ((long)mu * B);
    long mu0 = rem / B, k0 = rem % B;
    long muv = lp / B, kv = lp % B;
    a.C0[x] = mk<double>((muv == mu0 && kv == k0) ? 1.0 : 0.0, 0.0);
  }
  if (a.W0 && a.h1c0) {
    long long sidx = *a.step;
    double fv = (sidx < a.n_f) ? a.f[sidx] : 0.0;
    zd c = mk<double>(0.0, -a.dt * fv);  // -i dt f(t_n)
    // step layout [s'][a][s][b] with a = branch 0; H1 core 0 in builder layout [1][(2s'+s)][j]
    long ne = 4L * a.drive_D1;
    for (long x = tid; x < ne; x += stride) {
      int p = (int)(x / a.drive_D1), j = (int)(x % a.drive_D1);
      int so = p >> 1, si = p & 1;
      a.W0[(((long)so * B + 0) * 2 + si) * a.D1tot + a.drive_off + j] = cmul(c, a.h1c0[x]);
    }
  }
}
__global__ void k_step_begin(StepBeginArgs a) { step_begin_body(a); }
__global__ void k_step_begin_grp(const StepBeginArgs* __restrict__ a) { step_begin_body(a[blockIdx.y]); }

__global__ void k_step_end(StepEndArgs a) {
  if (a.count && threadIdx.x == 0 && blockIdx.x == 0) (*a.step)++;
}
__global__ void k_step_end_grp(const StepEndArgs* __restrict__ a) {
  const StepEndArgs x = a[blockIdx.y];
  if (x.count && threadIdx.x == 0 && blockIdx.x == 0) (*x.step)++;
}

// z_i = d_i for every bond (truncate-only pass has no zip-up)
__global__ void k_zip_from_state(int* d, int L) {
  int i = threadIdx.x;
  if (i <= L) d[L + 1 + i] = d[i];
}

// dst[x] = src[x] for x < c * d[a] * d[b]
__device__ void copy_body(const CopyArgs& c) {
  long n = dev_eval(c.cnt, c.d);
  for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < n; x += (long)gridDim.x * blockDim.x)
    c.dst[x] = c.src[x];
}
__global__ void k_copy(CopyArgs c) { copy_body(c); }
__global__ void k_copy_grp(const CopyArgs* __restrict__ c) { copy_body(c[blockIdx.y]); }

__global__ void k_sum_abs2(const zd* p, DimExpr cnt, const int* d, double* out) {
  __shared__ double sh[32];
  long n = dev_eval(cnt, d);
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

// builder layout [a][(2s'+s)][b] -> step layout [s'][a][s][b]
__global__ void k_to_step_layout(const zd* src, int Da, int Db, zd* dst) {
  long x = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long n = (long)Da * 4 * Db;
  if (x >= n) return;
  int a = (int)(x / (4L * Db));
  int rem = (int)(x % (4L * Db));
  int p = rem / Db, b = rem % Db;
  int so = p >> 1, si = p & 1;
  dst[(((long)so * Da + a) * 2 + si) * Db + b] = src[x];
}

// step layout [s'][a][s][b] -> builder layout [a][(2s'+s)][b], keeping only left index a0 (Da_out = 1)
__global__ void k_from_step_layout(const zd* src, int Da, int Db, int a0, zd* dst) {
  long x = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int Dout = a0 >= 0 ? 1 : Da;
  long n = (long)Dout * 4 * Db;
  if (x >= n) return;
  int a = (int)(x / (4L * Db));
  int rem = (int)(x % (4L * Db));
  int p = rem / Db, b = rem % Db;
  int so = p >> 1, si = p & 1;
  int as = a0 >= 0 ? a0 : a;
  dst[x] = src[(((long)so * Da + as) * 2 + si) * Db + b];
}

// drive coefficient rewrite alone (same formula as in k_step_begin)
__global__ void k_drive_rewrite(zd* W0, const zd* h1c0, int B, int D1tot, int drive_off, int drive_D1, const double* f,
                                long long n_f, const long long* step, double dt) {
  long long sidx = *step;
  double fv = (sidx < n_f) ? f[sidx] : 0.0;
  zd c = mk<double>(0.0, -dt * fv);
  long ne = 4L * drive_D1;
  for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < ne; x += (long)gridDim.x * blockDim.x) {
    int p = (int)(x / drive_D1), j = (int)(x % drive_D1);
    int so = p >> 1, si = p & 1;
    W0[(((long)so * B + 0) * 2 + si) * D1tot + drive_off + j] = cmul(c, h1c0[x]);
  }
}

__global__ void k_identity_core(zd* W) {
  // step layout [s'][a=1][s][b=1]: delta_{s's}
  int x = threadIdx.x;
  if (x < 4) W[x] = mk<double>((x == 0 || x == 3) ? 1.0 : 0.0, 0.0);
}

}  // namespace

// ------------------------------------------------------------------ launch helpers

static void prof_before(qlb_ctx* ctx, cudaStream_t sm, int kclass, cudaEvent_t* a) {
  *a = nullptr;
  if (!ctx->prof_on) return;
  if (ctx->ev_used + 2 > ctx->ev_pool.size()) {
    for (int i = 0; i < 256; i++) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ctx->ev_pool.push_back(e);
    }
  }
  *a = ctx->ev_pool[ctx->ev_used++];
  cudaEventRecord(*a, sm);
  (void)kclass;
}
static void prof_after(qlb_ctx* ctx, cudaStream_t sm, int kclass, cudaEvent_t a) {
  if (!ctx->prof_on || !a) return;
  cudaEvent_t b = ctx->ev_pool[ctx->ev_used++];
  cudaEventRecord(b, sm);
  ctx->prof_events.push_back({kclass, a, b});
}

#ifdef QLB_DEBUG_DUMP
// Debug builds only (compiled with -DQLB_DEBUG_DUMP): with QLB_DEBUG_DUMP=<file> in
// the environment, append the dims array, the error flags and the first entries of
// the output after every launch of an uncaptured step.
static FILE* debug_file() {
  static FILE* f = nullptr;
  static bool init = false;
  if (!init) {
    init = true;
    const char* p = getenv("QLB_DEBUG_DUMP");
    if (p && *p) f = fopen(p, "wb");
  }
  return f;
}
static void debug_dump(qlb_state* st, int tag, const void* out) {
  FILE* f = debug_file();
  if (!f) return;
  cudaStreamCaptureStatus cs;
  cudaStreamIsCapturing(st->stream, &cs);
  if (cs != cudaStreamCaptureStatusNone) return;
  cudaStreamSynchronize(st->stream);
  int n = 2 * st->L + 2;
  std::vector<int> d(n);
  cudaMemcpy(d.data(), st->d_dims, sizeof(int) * n, cudaMemcpyDeviceToHost);
  int err = 0;
  cudaMemcpy(&err, st->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  std::vector<zd> buf(64, mk<double>(0, 0));
  auto it = g_alloc_sizes().find(const_cast<void*>(out));
  size_t avail = it == g_alloc_sizes().end() ? 0 : it->second.first / sizeof(zd);
  cudaMemcpy(buf.data(), out, sizeof(zd) * std::min<size_t>(64, avail), cudaMemcpyDeviceToHost);
  fwrite(&tag, sizeof(int), 1, f);
  fwrite(&n, sizeof(int), 1, f);
  fwrite(d.data(), sizeof(int), n, f);
  fwrite(&err, sizeof(int), 1, f);
  fwrite(buf.data(), sizeof(zd), 64, f);
  fflush(f);
}
#else
static inline FILE* debug_file() { return nullptr; }
static inline void debug_dump(qlb_state*, int, const void*) {}
#endif

static qlb_status gemm(qlb_state* st, GemmDesc& g) {
  qlb_ctx* ctx = st->sys->ctx;
  if (!g.ws && st->Wsk && st->nWsk >= gemm_workspace_elems(gemm_grid_default())) g.ws = st->Wsk;
  // the mixed forms multiply in double-float (FP64 operands and results)
  if (st->prec != QLB_PREC_F64)
    g.df64 = ctx->opt.mixed_gemm >= 2 || (ctx->opt.mixed_gemm == 1 && g.kclass != QLB_K_GRAM);
  if (st->rec) {
    LaunchRec r;
    r.kind = (st->prec == QLB_PREC_TC && g.kclass == QLB_K_CONTRACT) ? REC_GEMM_TC : REC_GEMM;
    r.kclass = g.kclass;
    r.df = g.df64;
    r.g = g;
    r.g.dims = st->d_dims;
    r.g.split_grid = gemm_grid_default();
    r.err = st->d_err;
    r.dims = st->d_dims;
    st->rec->push_back(r);
    return QLB_OK;
  }
  cudaEvent_t a;
  prof_before(ctx, st->stream, g.kclass, &a);
  double* pf = ctx->prof_on ? ctx->d_prof + g.kclass : nullptr;
  // the tensor-core form runs the MPO application (the zip-up contractions) in
  // 3xTF32 on tcgen05; everything feeding a truncation decision stays FP64
  cudaError_t e = (st->prec == QLB_PREC_TC && g.kclass == QLB_K_CONTRACT)
                      ? launch_gemm_tc(g, st->d_dims, st->stream, st->d_err, pf)
                      : launch_gemm<double>(g, st->d_dims, st->stream, pf);
  prof_after(ctx, st->stream, g.kclass, a);
  if (e != cudaSuccess) {
    set_error(std::string("gemm launch: ") + cudaGetErrorString(e));
    return QLB_EDEVICE;
  }
  debug_dump(st, 1, g.C);
  return QLB_OK;
}

static qlb_status eig(qlb_state* st, EigDesc& e) {
  qlb_ctx* ctx = st->sys->ctx;
  e.solver_stats = ctx->d_solver;
  if (st->rec) {
    LaunchRec r;
    r.kind = REC_EIG;
    r.kclass = QLB_K_EIG;
    r.df = st->prec != QLB_PREC_F64;
    r.e = e;
    r.e.dims = st->d_dims;
    r.e.work = st->eigw;
    st->rec->push_back(r);
    return QLB_OK;
  }
  cudaEvent_t a;
  prof_before(ctx, st->stream, QLB_K_EIG, &a);
  double* pf = ctx->prof_on ? ctx->d_prof + QLB_K_EIG : nullptr;
  // the mixed form runs the same Jacobi in double-float on the FP32 pipes
  cudaError_t r = st->prec != QLB_PREC_F64 ? launch_eig<df64>(e, st->d_dims, st->stream, st->eigw, pf)
                                           : launch_eig<double>(e, st->d_dims, st->stream, st->eigw, pf);
  prof_after(ctx, st->stream, QLB_K_EIG, a);
  if (r != cudaSuccess) {
    set_error(std::string("eig launch: ") + cudaGetErrorString(r));
    return QLB_EDEVICE;
  }
  debug_dump(st, 2, e.out);
  return QLB_OK;
}

// A zip-up bond needs only an orthonormal basis of the range of M at the zip-up
// cutoff: the pivoted Gram-Schmidt basis first; the Jacobi solve behind it runs
// (through the gate) only when the basis reached the cap before the cutoff.
static qlb_status zip_range(qlb_state* st, EigDesc& e) {
  qlb_ctx* ctx = st->sys->ctx;
  if (!ctx->opt.zip_solver) return eig(st, e);
  e.solver_stats = ctx->d_solver;
  e.gate = st->d_gate;
  if (st->rec) {
    LaunchRec r;
    r.kind = REC_ZIPQR;
    r.kclass = QLB_K_EIG;
    r.df = st->prec != QLB_PREC_F64;
    r.e = e;
    r.e.dims = st->d_dims;
    r.e.work = st->eigw;
    st->rec->push_back(r);
    return eig(st, e);
  }
  cudaEvent_t a;
  prof_before(ctx, st->stream, QLB_K_EIG, &a);
  double* pf = ctx->prof_on ? ctx->d_prof + QLB_K_EIG : nullptr;
  cudaError_t r = st->prec != QLB_PREC_F64 ? launch_zipqr<df64>(e, st->d_dims, st->stream, st->eigw, pf)
                                           : launch_zipqr<double>(e, st->d_dims, st->stream, st->eigw, pf);
  prof_after(ctx, st->stream, QLB_K_EIG, a);
  if (r != cudaSuccess) {
    set_error(std::string("zip-up range basis launch: ") + cudaGetErrorString(r));
    return QLB_EDEVICE;
  }
  debug_dump(st, 3, e.out);
  return eig(st, e);
}

static qlb_status copy(qlb_state* st, zd* dst, const zd* src, DimExpr cnt, long max_n) {
  qlb_ctx* ctx = st->sys->ctx;
  const CopyArgs c{dst, src, cnt, st->d_dims};
  if (st->rec) {
    LaunchRec r;
    r.kind = REC_COPY;
    r.kclass = QLB_K_OTHER;
    r.c = c;
    r.grid_n = max_n;
    st->rec->push_back(r);
    return QLB_OK;
  }
  cudaEvent_t a;
  prof_before(ctx, st->stream, QLB_K_OTHER, &a);
  k_copy<<<nblk(max_n), 256, 0, st->stream>>>(c);
  prof_after(ctx, st->stream, QLB_K_OTHER, a);
  QLB_CUDA_TRY(cudaGetLastError());
  return QLB_OK;
}

static GemmDesc gdesc() {
  GemmDesc g{};
  g.sA1 = g.sB1 = g.sC1 = g.sA2 = g.sB2 = g.sC2 = dconst(0);
  g.nb1 = g.nb2 = dconst(1);
  g.nb_max = 1;
  g.opA = g.opB = OP_N;
  g.alpha_re = 1.0;
  g.alpha_im = 0.0;
  return g;
}

// ------------------------------------------------------------------ Kraus MPO

Kraus::~Kraus() {
  for (auto p : W) dev_free(nullptr, p);
  if (drive_core0) dev_free(nullptr, drive_core0);
}

static void kraus_clear(qlb_ctx* ctx, Kraus& K) {
  for (auto p : K.W) dev_free(ctx, p);
  K.W.clear();
  if (K.drive_core0) dev_free(ctx, K.drive_core0);
  K.drive_core0 = nullptr;
  K.D.clear();
  K.driven = false;
  K.dt = -1;
  K.version = -1;
}

static qlb_status kraus_from_mpo(qlb_ctx* ctx, const Mpo& S, Kraus& K) {
  K.L = S.L;
  K.D = S.D;
  K.B = S.D[0];
  K.W.assign(S.L, nullptr);
  for (int i = 0; i < S.L; i++) {
    long n = (long)S.D[i] * 4 * S.D[i + 1];
    qlb_status st = dev_alloc(ctx, (void**)&K.W[i], sizeof(zd) * n);
    if (st) return st;
    k_to_step_layout<<<nblk(n), 256, 0, ctx->stream>>>(S.core[i], S.D[i], S.D[i + 1], K.W[i]);
  }
  QLB_CUDA_TRY(cudaGetLastError());
  return QLB_OK;
}

qlb_status build_identity_kraus(qlb_state* st) {
  qlb_ctx* ctx = st->sys->ctx;
  if (st->kraus_id.dt == 0.0 && st->kraus_id.version == -2) return QLB_OK;
  kraus_clear(ctx, st->kraus_id);
  Kraus& K = st->kraus_id;
  K.L = st->L;
  K.B = 1;
  K.D.assign(st->L + 1, 1);
  K.W.assign(st->L, nullptr);
  for (int i = 0; i < st->L; i++) {
    qlb_status s = dev_alloc(ctx, (void**)&K.W[i], 4 * sizeof(zd));
    if (s) return s;
    k_identity_core<<<1, 32, 0, ctx->stream>>>(K.W[i]);
  }
  QLB_CUDA_TRY(cudaGetLastError());
  K.dt = 0.0;
  K.version = -2;
  K.unstable_factor = 0.0;
  return QLB_OK;
}

// K_0 = U_1 = 1 - i h H_eff, H_eff = H0 - (i/2) sum_k L_k^dag L_k (Sec. V.B), K_k = sqrt(h) L_k;
// stacked with branch k on the left boundary and jointly recompressed.  With a
// drive the H1 block is appended uncompressed on branch 0 and its core 0 is
// rewritten every step with -i h f(t_n).
// Device copy of a Kraus MPO (each state owns its copy: the drive rewrites core 0).
static qlb_status kraus_copy(qlb_ctx* ctx, const Kraus& src, Kraus& dst) {
  kraus_clear(ctx, dst);
  dst.dt = src.dt;
  dst.version = src.version;
  dst.B = src.B;
  dst.L = src.L;
  dst.D = src.D;
  dst.driven = src.driven;
  dst.drive_off = src.drive_off;
  dst.drive_D1 = src.drive_D1;
  dst.unstable_factor = src.unstable_factor;
  dst.W.assign(src.L, nullptr);
  for (int i = 0; i < src.L; i++) {
    size_t b = sizeof(zd) * (size_t)src.D[i] * 4 * src.D[i + 1];
    qlb_status s = dev_alloc(ctx, (void**)&dst.W[i], b);
    if (s) return s;
    QLB_CUDA_TRY(cudaMemcpyAsync(dst.W[i], src.W[i], b, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  if (src.drive_core0) {
    size_t b = sizeof(zd) * 4 * (size_t)src.drive_D1;
    qlb_status s = dev_alloc(ctx, (void**)&dst.drive_core0, b);
    if (s) return s;
    QLB_CUDA_TRY(cudaMemcpyAsync(dst.drive_core0, src.drive_core0, b, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  QLB_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return QLB_OK;
}

// Product of two terms of operators, mode by mode: out = scale * op(a) * b with
// op(a) = a or a^dag.  Dense products are appended to tmp (freed by the caller);
// factors that need no product are borrowed.  Recipes (keys) compose so that the
// context's MPO cache recognises repeated products of built-in factors.
static qlb_status term_mul(qlb_system* sys, const DevTerm& a, bool dag_a, const DevTerm& b, zd scale, DevTerm& out,
                           std::vector<zd*>& tmp) {
  qlb_ctx* ctx = sys->ctx;
  qlb_status s;
  out.coeff = cmul(cmul(dag_a ? cconj(a.coeff) : a.coeff, b.coeff), scale);
  out.fac.assign(sys->M, nullptr);
  out.key.assign(sys->M, "");
  for (int m = 0; m < sys->M; m++) {
    int N = 1 << sys->R[m];
    const zd* A = a.fac[m];
    const zd* Bm = b.fac[m];
    if (!A && !Bm) continue;
    const std::string& ka = a.key[m];
    const std::string& kb = b.key[m];
    if (!A)
      out.key[m] = kb;
    else if (!Bm)
      out.key[m] = ka.empty() ? std::string() : (dag_a ? "dag(" + ka + ")" : ka);
    else if (!ka.empty() && !kb.empty())
      out.key[m] = (dag_a ? "dag(" + ka + ")" : "(" + ka + ")") + "*(" + kb + ")";
    if (!A) {
      out.fac[m] = const_cast<zd*>(Bm);
      continue;
    }
    if (!Bm && !dag_a) {
      out.fac[m] = const_cast<zd*>(A);
      continue;
    }
    zd* P = nullptr;
    if (Bm) {
      if ((s = dense_mul(ctx, A, dag_a ? OP_C : OP_N, Bm, N, &P))) return s;
    } else {  // A^dag alone
      zd* I = nullptr;
      qlb_factor f{m, QLB_F_ID, 1, 0.0, nullptr};
      if ((s = make_factor(ctx, N, f, &I))) return s;
      s = dense_mul(ctx, A, OP_C, I, N, &P);
      dev_free(ctx, I);
      if (s) return s;
    }
    tmp.push_back(P);
    out.fac[m] = P;
  }
  return QLB_OK;
}

static qlb_status build_kraus_fresh(qlb_state* st, double dt);

qlb_status build_kraus(qlb_state* st, double dt) {
  qlb_system* sys = st->sys;
  qlb_ctx* ctx = sys->ctx;
  if (st->kraus.dt == dt && st->kraus.version == sys->version) return QLB_OK;
  if (!sys->H0 && sys->jumps.empty()) {
    set_error("system has neither a Hamiltonian nor jump operators");
    return QLB_ESTATE;
  }
  Kraus* t = sys->kraus_tmpl;
  if (t && t->dt == dt && t->version == sys->version) return kraus_copy(ctx, *t, st->kraus);
  qlb_status s = build_kraus_fresh(st, dt);
  if (s) return s;
  if (!t) t = sys->kraus_tmpl = new Kraus();
  return kraus_copy(ctx, st->kraus, *t);
}

static qlb_status build_kraus_fresh(qlb_state* st, double dt) {
  qlb_system* sys = st->sys;
  qlb_ctx* ctx = sys->ctx;
  kraus_clear(ctx, st->kraus);
  qlb_status s;
  if (sys->order == 2 && (sys->H1 || sys->jumps.size() > 6)) {
    set_error("the second-order scheme needs H1 == NULL and at most 6 jump operators");
    return QLB_EINVAL;
  }
  // H_eff = H0 - (i/2) sum_k L_k^dag L_k (Sec. V.B), L^dag L formed term by term
  std::vector<zd*> tmp;  // dense products made for this build
  struct Tmp {
    qlb_ctx* c;
    std::vector<zd*>& v;
    ~Tmp() {
      for (auto p : v) dev_free(c, p);
    }
  } tmp_guard{ctx, tmp};
  std::vector<DevTerm> heff;
  if (sys->H0)
    for (auto& t : sys->H0->terms) heff.push_back(t);
  double gamma_bound = 0.0;
  for (const qlb_op* L : sys->jumps) {
    gamma_bound += L->inf_norm_bound * L->inf_norm_bound;
    for (auto& ta : L->terms)
      for (auto& tb : L->terms) {
        DevTerm u;
        if ((s = term_mul(sys, ta, true, tb, mk<double>(0.0, -0.5), u, tmp))) return s;
        heff.push_back(u);
      }
  }
  DevTerm id;
  id.coeff = mk<double>(1.0, 0.0);
  id.fac.assign(sys->M, nullptr);
  id.key.assign(sys->M, "");
  // U_1 = 1 - i h H_eff
  std::vector<DevTerm> u1 = {id};
  for (auto& t : heff) {
    DevTerm u = t;
    u.coeff = cmul(t.coeff, mk<double>(0.0, -dt));
    u1.push_back(u);
  }
  // Kraus operators of the scheme, branch k on the left boundary (Sec. V.B):
  //   order 1: U_1, sqrt(h) L_k
  //   order 2: U_1' = U_1 - (h^2/2) H_eff^2, sqrt(h/2) U_1 L_k, sqrt(h/2) L_k U_1,
  //            (h/sqrt 2) L_j L_k   (K = U' + (h/2)(U L + L U) + (h^2/2) L^2)
  std::vector<std::vector<DevTerm>> branches;
  const size_t l = sys->jumps.size();
  if (sys->order == 1) {
    branches.push_back(u1);  // the jump branches reuse the operators' own MPOs below
  } else {
    std::vector<DevTerm> u1p = u1;
    for (auto& a : heff)
      for (auto& b : heff) {
        DevTerm u;
        if ((s = term_mul(sys, a, false, b, mk<double>(-0.5 * dt * dt, 0.0), u, tmp))) return s;
        u1p.push_back(u);
      }
    branches.push_back(u1p);
    const double r = std::sqrt(0.5 * dt);
    for (int side = 0; side < 2; side++)
      for (size_t k = 0; k < l; k++) {
        std::vector<DevTerm> b;
        for (auto& x : u1)
          for (auto& y : sys->jumps[k]->terms) {
            DevTerm u;
            if ((s = side == 0 ? term_mul(sys, x, false, y, mk<double>(r, 0.0), u, tmp)
                               : term_mul(sys, y, false, x, mk<double>(r, 0.0), u, tmp)))
              return s;
            b.push_back(u);
          }
        branches.push_back(b);
      }
    for (size_t j = 0; j < l; j++)
      for (size_t k = 0; k < l; k++) {
        std::vector<DevTerm> b;
        for (auto& x : sys->jumps[j]->terms)
          for (auto& y : sys->jumps[k]->terms) {
            DevTerm u;
            if ((s = term_mul(sys, x, false, y, mk<double>(dt / std::sqrt(2.0), 0.0), u, tmp))) return s;
            b.push_back(u);
          }
        branches.push_back(b);
      }
  }
  const int B = sys->order == 1 ? (int)(1 + l) : (int)branches.size();
  std::vector<Mpo> bm(B);
  struct Parts {
    qlb_ctx* c;
    std::vector<Mpo>& v;
    ~Parts() {
      for (auto& m : v) mpo_clear(c, m);
    }
  } parts_guard{ctx, bm};
  std::vector<const Mpo*> parts;
  std::vector<int> rows;
  for (int k = 0; k < B; k++) {
    if (k < (int)branches.size()) {
      if ((s = mpo_from_terms(sys, branches[k], 1e-30, 0, bm[k]))) return s;
    } else {
      if ((s = mpo_copy(ctx, sys->jumps[k - 1]->mpo, bm[k]))) return s;
      if ((s = mpo_scale(ctx, bm[k], mk<double>(std::sqrt(dt), 0.0)))) return s;
    }
    parts.push_back(&bm[k]);
    rows.push_back(k);
  }
  Mpo S;
  if ((s = mpo_stack(ctx, parts, rows, B, S))) return s;
  if ((s = mpo_compress(ctx, S, 1e-30, 0))) return s;
  Kraus& K = st->kraus;
  if (sys->H1) {
    // append the H1 block on branch 0
    Mpo H1c;
    if ((s = mpo_copy(ctx, sys->H1->mpo, H1c))) return s;
    std::vector<const Mpo*> p2 = {&S, &H1c};
    Mpo S2;
    if ((s = mpo_stack(ctx, p2, {0, 0}, B, S2))) return s;
    K.driven = true;
    K.drive_off = S.D[1];
    K.drive_D1 = H1c.D[1];
    long n0 = 4L * H1c.D[1];
    if ((s = dev_alloc(ctx, (void**)&K.drive_core0, sizeof(zd) * n0))) return s;
    QLB_CUDA_TRY(cudaMemcpyAsync(K.drive_core0, H1c.core[0], sizeof(zd) * n0, cudaMemcpyDeviceToDevice, ctx->stream));
    // H1 core 0 starts at zero in the stacked MPO (rewritten each step)
    mpo_clear(ctx, H1c);
    mpo_clear(ctx, S);
    if ((s = kraus_from_mpo(ctx, S2, K))) return s;
    mpo_clear(ctx, S2);
  } else {
    if ((s = kraus_from_mpo(ctx, S, K))) return s;
    mpo_clear(ctx, S);
  }
  QLB_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  K.dt = dt;
  K.version = sys->version;
  K.unstable_factor = dt * gamma_bound;
  return QLB_OK;
}

// ------------------------------------------------------------------ buffers

static qlb_status realloc_buf(qlb_ctx* ctx, zd** p, size_t* have, size_t need) {
  if (*p && *have >= need) return QLB_OK;
  dev_free(ctx, *p);
  *p = nullptr;
  *have = 0;
  qlb_status s = dev_alloc(ctx, (void**)p, sizeof(zd) * std::max<size_t>(need, 1));
  if (s) return s;
  *have = need;
  return QLB_OK;
}

struct Caps {
  std::vector<int> dcap, zcap;
  std::vector<int> hd;  // host mirror of caps in the dims layout
};

static Caps compute_caps(const qlb_state* st, const std::vector<int>& cur, const Kraus& K) {
  const int L = st->L;
  Caps c;
  c.dcap.assign(L + 1, 1);
  c.zcap.assign(L + 1, 1);
  // the purification rank never exceeds the Hilbert-space dimension 2^L
  c.dcap[0] = std::max(std::min<long>(st->cap_mu, 1L << std::min(L, 30)), (long)cur[0]);
  for (int i = 1; i < L; i++) {
    long right = 1L << std::min(L - i, 30);
    long left = (long)st->cap_mu << std::min(i, 30);
    long v = std::min<long>({(long)st->cap_chi, right, left});
    c.dcap[i] = (int)std::max<long>(v, cur[i]);
  }
  c.zcap[0] = c.dcap[0] * K.B;
  // zip-up bond i: rank(M) <= min(2 z_{i-1}, d_i D_i).  It is not bounded by the
  // right Hilbert dimension 2^(L-i): the right environment of the zip-up holds
  // the MPO and is no isometry, so M can need more columns than the final Schmidt rank.
  const qlb_options& o = st->sys->ctx->opt;
  const long zip_cap = o.zip_chi_max > 0 ? std::max(o.zip_chi_max, st->cap_chi) : st->cap_chi;
  for (int i = 1; i < L; i++) {
    long v = std::min<long>({zip_cap, 2L * c.zcap[i - 1], (long)c.dcap[i] * K.D[i]});
    c.zcap[i] = (int)std::max<long>(v, 1);
    c.zcap[i] = std::max(c.zcap[i], cur[i]);  // truncate-only pass: z_i = d_i
  }
  c.hd.assign(2 * L + 2, 1);
  for (int i = 0; i <= L; i++) {
    c.hd[SB(i)] = c.dcap[i];
    c.hd[ZB(st, i)] = c.zcap[i];
  }
  return c;
}

qlb_status plan_buffers(qlb_state* st, const Kraus& K) {
  qlb_ctx* ctx = st->sys->ctx;
  const int L = st->L;
  std::vector<int> cur;
  qlb_status s;
  if ((s = read_dims(st, cur))) return s;
  Caps c = compute_caps(st, cur, K);
  const std::vector<int>& D = K.D;
  const int B = K.B;
  size_t nX = 1, nM = 1, nC = 1, nG = 1, nT = 1;
  int n_eig = 1;
  nC = (size_t)c.zcap[0] * c.dcap[0] * B;
  for (int i = 0; i < L; i++) {
    nX = std::max(nX, (size_t)c.zcap[i] * D[i] * 2 * c.dcap[i + 1]);
    nM = std::max(nM, (size_t)2 * c.zcap[i] * c.dcap[i + 1] * D[i + 1]);
    if (i + 1 <= L) nC = std::max(nC, (size_t)c.zcap[i + 1] * c.dcap[i + 1] * D[i + 1]);
    if (i < L - 1) {
      nG = std::max(nG, (size_t)4 * c.zcap[i] * c.zcap[i]);
      n_eig = std::max(n_eig, 2 * c.zcap[i]);
    }
    if (i >= 1) {
      nG = std::max(nG, (size_t)4 * c.dcap[i + 1] * c.dcap[i + 1]);
      n_eig = std::max(n_eig, 2 * c.dcap[i + 1]);
      nT = std::max({nT, (size_t)c.dcap[i] * 2 * c.dcap[i + 1], (size_t)c.zcap[i] * c.dcap[i],
                     (size_t)2 * c.zcap[i - 1] * c.dcap[i], (size_t)2 * c.zcap[i] * c.dcap[i + 1]});
    }
  }
  nG = std::max(nG, (size_t)c.zcap[0] * c.zcap[0]);
  n_eig = std::max(n_eig, c.zcap[0]);
  nT = std::max({nT, (size_t)c.zcap[0] * c.dcap[0], (size_t)c.dcap[0] * 2 * c.dcap[1], (size_t)c.zcap[0] * 2 * c.dcap[1]});
  if (n_eig > 512) {
    std::string dims;
    for (int v : cur) dims += " " + std::to_string(v);
    set_error("a truncation would need an eigen-solve of size " + std::to_string(n_eig) + " (> 512); bond dims" + dims);
    return QLB_EINVAL;
  }
  if ((s = realloc_buf(ctx, &st->X, &st->nX, nX))) return s;
  if ((s = realloc_buf(ctx, &st->Mb, &st->nM, nM))) return s;
  {
    size_t c1 = st->nC, c2 = st->nC;
    if ((s = realloc_buf(ctx, &st->Cin, &c1, nC))) return s;
    if ((s = realloc_buf(ctx, &st->Cout, &c2, nC))) return s;
    st->nC = std::max(st->nC, nC);
  }
  if ((s = realloc_buf(ctx, &st->G, &st->nG, nG))) return s;
  size_t t1 = st->nT, t2 = st->nT, t3 = st->nT;
  if ((s = realloc_buf(ctx, &st->T1, &t1, nT))) return s;
  if ((s = realloc_buf(ctx, &st->T2, &t2, nT))) return s;
  if ((s = realloc_buf(ctx, &st->T3, &t3, nT))) return s;
  st->nT = std::max(st->nT, nT);
  // every GEMM of the step runs on the work-distributed grid with this workspace;
  // the zip-up Grams take the tuned cap on their K split when the table has one
  st->gram_split.assign(L, 1);
  for (int i = 0; i + 1 < L; i++) {
    const long mm = 2L * c.zcap[i], kk = (long)c.dcap[i + 1] * D[i + 1];
    st->gram_split[i] = gram_splitk(ctx, mm, kk);
  }
  {
    zd* before = st->Wsk;
    if ((s = realloc_buf(ctx, &st->Wsk, &st->nWsk, gemm_workspace_elems(gemm_grid_default())))) return s;
    if (st->Wsk != before) QLB_CUDA_TRY(cudaMemsetAsync(st->Wsk, 0, sizeof(zd) * st->nWsk, st->stream));
  }
  size_t new_ew = eig_workspace_elems(n_eig);
  if (ctx->opt.zip_solver) new_ew = std::max(new_ew, zipqr_workspace_elems(n_eig));
  if ((s = realloc_buf(ctx, &st->eigw, &st->nEw, new_ew))) return s;
  if (!st->d_lam) {
    if ((s = dev_alloc(ctx, (void**)&st->d_lam, sizeof(double) * 1024))) return s;
  }
  if (!st->d_gate) {
    if ((s = dev_alloc(ctx, (void**)&st->d_gate, sizeof(int)))) return s;
  }
  // sites: grow keeping their content
  for (int i = 0; i < L; i++) {
    size_t need = (size_t)std::max(c.dcap[i], c.zcap[i]) * 2 * std::max(c.dcap[i + 1], c.zcap[i + 1]);
    if (need > st->site_cap[i]) {
      zd* p = nullptr;
      if ((s = dev_alloc(ctx, (void**)&p, sizeof(zd) * need))) return s;
      size_t have = (size_t)cur[i] * 2 * cur[i + 1];
      if (st->site[i] && have)
        QLB_CUDA_TRY(cudaMemcpyAsync(p, st->site[i], sizeof(zd) * have, cudaMemcpyDeviceToDevice, st->stream));
      dev_free(ctx, st->site[i]);
      st->site[i] = p;
      st->site_cap[i] = need;
    }
  }
  // grid bounds only grow, so a graph captured earlier stays valid for smaller plans
  if (st->cap_state.size() == c.hd.size())
    for (size_t j = 0; j < c.hd.size(); j++) c.hd[j] = std::max(c.hd[j], st->cap_state[j]);
  st->cap_state = c.hd;
  st->plan_key++;
  QLB_CUDA_TRY(cudaStreamSynchronize(st->stream));
  return QLB_OK;
}

// ------------------------------------------------------------------ the step

static qlb_status enqueue_compress(qlb_state* st, const std::vector<int>& hd) {
  const int L = st->L;
  qlb_ctx* ctx = st->sys->ctx;
  const qlb_options& o = ctx->opt;
  qlb_status s;
  auto cap = [&](int idx) { return hd[idx]; };
  for (int i = L - 1; i >= 1; i--) {
    // G = M^dag M, M = A_i as [z_i] x [(s, d_{i+1})]
    GemmDesc g = gdesc();
    g.kclass = QLB_K_GRAM;
    g.A = st->site[i];
    g.B = st->site[i];
    g.C = st->G;
    g.m = g.n = dvar(SB(i + 1), 2);
    g.k = dvar(ZB(st, i));
    g.opA = OP_C;
    g.lda = dvar(SB(i + 1), 2);
    g.ldb = dvar(SB(i + 1), 2);
    g.ldc = dvar(SB(i + 1), 2);
    g.m_max = g.n_max = 2 * cap(SB(i + 1));
    if ((s = gemm(st, g))) return s;
    EigDesc e{};
    e.G = st->G;
    e.lam = nullptr;
    e.n = dvar(SB(i + 1), 2);
    e.n_max = 2 * cap(SB(i + 1));
    e.out = st->T1;
    e.out_mode = 1;
    e.dim_out = SB(i);
    e.tol = st->tol;
    e.cap = dconst(std::min(st->chi_max, cap(SB(i))));
    e.gap = o.degeneracy_gap;
    e.max_sweeps = o.max_sweeps;
    e.disc_stat = st->d_stats + 2;
    e.err = st->d_err;
    if ((s = eig(st, e))) return s;
    // US = M V_k  (V_k = T1^dag)
    g = gdesc();
    g.kclass = QLB_K_APPLY;
    g.A = st->site[i];
    g.B = st->T1;
    g.C = st->T2;
    g.m = dvar(ZB(st, i));
    g.n = dvar(SB(i));
    g.k = dvar(SB(i + 1), 2);
    g.opB = OP_C;
    g.lda = dvar(SB(i + 1), 2);
    g.ldb = dvar(SB(i + 1), 2);
    g.ldc = dvar(SB(i));
    g.m_max = cap(ZB(st, i));
    g.n_max = cap(SB(i));
    if ((s = gemm(st, g))) return s;
    if ((s = copy(st, st->site[i], st->T1, dvar2(SB(i), SB(i + 1), 2), (long)cap(SB(i)) * 2 * cap(SB(i + 1)))))
      return s;
    // A_{i-1} <- A_{i-1} US
    g = gdesc();
    g.kclass = QLB_K_APPLY;
    g.A = st->site[i - 1];
    g.B = st->T2;
    g.C = st->T3;
    g.m = dvar(ZB(st, i - 1), 2);
    g.n = dvar(SB(i));
    g.k = dvar(ZB(st, i));
    g.lda = dvar(ZB(st, i));
    g.ldb = dvar(SB(i));
    g.ldc = dvar(SB(i));
    g.m_max = 2 * cap(ZB(st, i - 1));
    g.n_max = cap(SB(i));
    if ((s = gemm(st, g))) return s;
    if ((s = copy(st, st->site[i - 1], st->T3, dvar2(ZB(st, i - 1), SB(i), 2),
                  (long)2 * cap(ZB(st, i - 1)) * cap(SB(i)))))
      return s;
  }
  // purification rank: G = A_0 A_0^dag over mu' = z_0
  {
    GemmDesc g = gdesc();
    g.kclass = QLB_K_GRAM;
    g.A = st->site[0];
    g.B = st->site[0];
    g.C = st->G;
    g.m = g.n = dvar(ZB(st, 0));
    g.k = dvar(SB(1), 2);
    g.opB = OP_C;
    g.lda = g.ldb = dvar(SB(1), 2);
    g.ldc = dvar(ZB(st, 0));
    g.m_max = g.n_max = cap(ZB(st, 0));
    if ((s = gemm(st, g))) return s;
    EigDesc e{};
    e.G = st->G;
    e.lam = st->d_lam;
    e.n = dvar(ZB(st, 0));
    e.n_max = cap(ZB(st, 0));
    e.out = st->T1;
    e.out_mode = 0;
    e.dim_out = SB(0);
    e.tol = st->tol;
    e.cap = dconst(std::min(st->chi_mu_max, cap(SB(0))));
    e.gap = o.degeneracy_gap;
    e.max_sweeps = o.max_sweeps;
    e.kept_weight = st->d_stats + 0;
    e.total_weight = st->d_stats + 1;
    e.err = st->d_err;
    if ((s = eig(st, e))) return s;
    g = gdesc();
    g.kclass = QLB_K_APPLY;
    g.A = st->T1;
    g.B = st->site[0];
    g.C = st->T2;
    g.m = dvar(SB(0));
    g.n = dvar(SB(1), 2);
    g.k = dvar(ZB(st, 0));
    g.opA = OP_C;
    g.lda = dvar(SB(0));
    g.ldb = dvar(SB(1), 2);
    g.ldc = dvar(SB(1), 2);
    g.alpha_scale = st->d_stats + 0;
    g.alpha_scale_rsqrt = 1;
    g.m_max = cap(SB(0));
    g.n_max = 2 * cap(SB(1));
    if ((s = gemm(st, g))) return s;
    if ((s = copy(st, st->site[0], st->T2, dvar2(SB(0), SB(1), 2), (long)cap(SB(0)) * 2 * cap(SB(1))))) return s;
  }
  return QLB_OK;
}

qlb_status enqueue_step(qlb_state* st, const Kraus& K, bool count_step) {
  const int L = st->L;
  qlb_ctx* ctx = st->sys->ctx;
  const qlb_options& o = ctx->opt;
  const std::vector<int>& hd = st->cap_state;
  auto cap = [&](int idx) { return hd[idx]; };
  qlb_status s;
  {
    long n0 = (long)cap(ZB(st, 0)) * cap(SB(0)) * K.B;
    const StepBeginArgs ba{st->d_dims,   L,         K.B,         st->Cin,         (long)st->nC,
                           K.driven ? K.W[0] : nullptr,          K.driven ? K.drive_core0 : nullptr,
                           K.D[1],       K.drive_off, K.drive_D1, st->sys->d_f,    st->sys->n_f,
                           st->d_step,   K.dt,      st->d_stats};
    if (st->rec) {
      LaunchRec r;
      r.kind = REC_BEGIN;
      r.kclass = QLB_K_OTHER;
      r.b = ba;
      r.grid_n = std::max<long>(n0, 4L * K.drive_D1);
      st->rec->push_back(r);
    } else {
      cudaEvent_t a;
      prof_before(ctx, st->stream, QLB_K_OTHER, &a);
      k_step_begin<<<nblk(n0), 256, 0, st->stream>>>(ba);
      prof_after(ctx, st->stream, QLB_K_OTHER, a);
      QLB_CUDA_TRY(cudaGetLastError());
    }
  }
  zd* Cin = st->Cin;
  zd* Cout = st->Cout;
  for (int i = 0; i < L; i++) {
    const int Dl = K.D[i], Dr = K.D[i + 1];
    // stage 1: X_l'[a][(s,r)] = sum_l C_l'[l][a] A[l][(s,r)]
    GemmDesc g = gdesc();
    g.kclass = QLB_K_CONTRACT;
    g.A = Cin;
    g.B = st->site[i];
    g.C = st->X;
    g.m = dconst(Dl);
    g.n = dvar(SB(i + 1), 2);
    g.k = dvar(SB(i));
    g.opA = OP_T;
    g.lda = dconst(Dl);
    g.ldb = dvar(SB(i + 1), 2);
    g.ldc = dvar(SB(i + 1), 2);
    g.sA1 = dvar(SB(i), Dl);
    g.sC1 = dvar(SB(i + 1), 2 * Dl);
    g.nb1 = dvar(ZB(st, i));
    g.m_max = Dl;
    g.n_max = 2 * cap(SB(i + 1));
    g.nb_max = cap(ZB(st, i));
    if ((s = gemm(st, g))) return s;
    // stage 2: M[(l',s')][(r,b)] = sum_{a,s} X_l'[(a,s)][r] W_s'[(a,s)][b]
    zd* Mdst = (i == L - 1) ? st->site[L - 1] : st->Mb;
    g = gdesc();
    g.kclass = QLB_K_CONTRACT;
    g.A = st->X;
    g.B = K.W[i];
    g.C = Mdst;
    g.m = dvar(SB(i + 1));
    g.n = dconst(Dr);
    g.k = dconst(2 * Dl);
    g.opA = OP_T;
    g.lda = dvar(SB(i + 1));
    g.ldb = dconst(Dr);
    g.ldc = dconst(Dr);
    g.sA1 = dvar(SB(i + 1), 2 * Dl);
    g.sB2 = dconst(Dl * 2 * Dr);
    g.sC1 = dvar(SB(i + 1), 2 * Dr);
    g.sC2 = dvar(SB(i + 1), Dr);
    g.nb1 = dvar(ZB(st, i));
    g.nb2 = dconst(2);
    g.m_max = cap(SB(i + 1));
    g.n_max = Dr;
    g.nb_max = 2 * cap(ZB(st, i));
    if ((s = gemm(st, g))) return s;
    if (i == L - 1) break;
    // Gram G = M M^dag  ((2 z_i) x (2 z_i), K = d_{i+1} Dr)
    g = gdesc();
    g.kclass = QLB_K_GRAM;
    g.A = st->Mb;
    g.B = st->Mb;
    g.C = st->G;
    g.m = g.n = dvar(ZB(st, i), 2);
    g.k = dvar(SB(i + 1), Dr);
    g.opB = OP_C;
    g.lda = g.ldb = dvar(SB(i + 1), Dr);
    g.ldc = dvar(ZB(st, i), 2);
    g.m_max = g.n_max = 2 * cap(ZB(st, i));
    if (i < (int)st->gram_split.size() && st->gram_split[i] >= 1) g.ksplit = st->gram_split[i];
    if ((s = gemm(st, g))) return s;
    EigDesc e{};
    e.G = st->G;
    e.n = dvar(ZB(st, i), 2);
    e.n_max = 2 * cap(ZB(st, i));
    e.out = st->site[i];
    e.out_mode = 0;
    e.dim_out = ZB(st, i + 1);
    e.tol = st->tol * o.zip_tol_factor;
    const int zc = o.zip_chi_max > 0 ? std::max(o.zip_chi_max, st->chi_max) : st->chi_max;
    e.cap = dconst(std::min(zc, cap(ZB(st, i + 1))));
    e.gap = o.degeneracy_gap;
    e.max_sweeps = o.max_sweeps;
    e.err = st->d_err;
    if ((s = zip_range(st, e))) return s;
    // carry C' = U^dag M  -> [k][(r, b)]
    g = gdesc();
    g.kclass = QLB_K_APPLY;
    g.A = st->site[i];
    g.B = st->Mb;
    g.C = Cout;
    g.m = dvar(ZB(st, i + 1));
    g.n = dvar(SB(i + 1), Dr);
    g.k = dvar(ZB(st, i), 2);
    g.opA = OP_C;
    g.lda = dvar(ZB(st, i + 1));
    g.ldb = dvar(SB(i + 1), Dr);
    g.ldc = dvar(SB(i + 1), Dr);
    g.m_max = cap(ZB(st, i + 1));
    g.n_max = cap(SB(i + 1)) * Dr;
    if ((s = gemm(st, g))) return s;
    std::swap(Cin, Cout);
  }
  if ((s = enqueue_compress(st, hd))) return s;
  {
    const StepEndArgs ea{st->d_step, count_step ? 1 : 0};
    if (st->rec) {
      LaunchRec r;
      r.kind = REC_END;
      r.kclass = QLB_K_OTHER;
      r.x = ea;
      st->rec->push_back(r);
    } else {
      cudaEvent_t a;
      prof_before(ctx, st->stream, QLB_K_OTHER, &a);
      k_step_end<<<1, 32, 0, st->stream>>>(ea);
      prof_after(ctx, st->stream, QLB_K_OTHER, a);
      QLB_CUDA_TRY(cudaGetLastError());
    }
  }
  return QLB_OK;
}

qlb_status read_dims(qlb_state* st, std::vector<int>& d) {
  qlb_ctx* ctx = st->sys->ctx;
  d.assign(2 * st->L + 2, 0);
  QLB_CUDA_TRY(cudaMemcpyAsync(d.data(), st->d_dims, sizeof(int) * d.size(), cudaMemcpyDeviceToHost, st->stream));
  QLB_CUDA_TRY(cudaStreamSynchronize(st->stream));
  return QLB_OK;
}

qlb_status run_steps(qlb_state* st, int64_t n, bool sync) {
  qlb_ctx* ctx = st->sys->ctx;
  qlb_status s;
  if (n <= 0) return QLB_OK;
  if (ctx->prof_on || debug_file()) {
    for (int64_t k = 0; k < n; k++)
      if ((s = enqueue_step(st, st->kraus, true))) return s;
  } else {
    if (!st->graph || st->graph_key != st->plan_key) {
      if (st->graph) cudaGraphExecDestroy(st->graph);
      st->graph = nullptr;
      cudaGraph_t gr;
      QLB_CUDA_TRY(cudaStreamBeginCapture(st->stream, cudaStreamCaptureModeThreadLocal));
      s = enqueue_step(st, st->kraus, true);
      cudaError_t e = cudaStreamEndCapture(st->stream, &gr);
      if (s) {
        if (e == cudaSuccess) cudaGraphDestroy(gr);
        return s;
      }
      QLB_CUDA_TRY(e);
      e = cudaGraphInstantiate(&st->graph, gr, 0);
      cudaGraphDestroy(gr);
      QLB_CUDA_TRY(e);
      st->graph_key = st->plan_key;
    }
    for (int64_t k = 0; k < n; k++) QLB_CUDA_TRY(cudaGraphLaunch(st->graph, st->stream));
  }
  st->host_steps += n;
  if (!sync) return QLB_OK;
  QLB_CUDA_TRY(cudaStreamSynchronize(st->stream));
  return check_flags(st);
}

// The state's device error flags and trace after its work has completed.
qlb_status check_flags(qlb_state* st) {
  int err = 0;
  QLB_CUDA_TRY(cudaMemcpy(&err, st->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    QLB_CUDA_TRY(cudaMemset(st->d_err, 0, sizeof(int)));
    if (err & 4) {
      set_error("a bounded wait of the tensor-core contraction gave up");
      return QLB_ETIMEOUT;
    }
    if (err & 2) {
      set_error("non-finite values met in a truncation");
      return QLB_ENONFINITE;
    }
    set_error("a Jacobi eigen-solve hit its sweep limit");
    return QLB_ENOTCONV;
  }
  double stats[2];
  QLB_CUDA_TRY(cudaMemcpy(stats, st->d_stats, sizeof(stats), cudaMemcpyDeviceToHost));
  if (!std::isfinite(stats[1])) {
    set_error("non-finite trace");
    return QLB_ENONFINITE;
  }
  return QLB_OK;
}

// Truncate-only pass: one sweep with the identity Kraus MPO, then the checks.
qlb_status truncate_pass(qlb_state* st) {
  qlb_status s;
  if ((s = build_identity_kraus(st))) return s;
  if ((s = plan_buffers(st, st->kraus_id))) return s;
  if ((s = enqueue_step(st, st->kraus_id, false))) return s;
  qlb_ctx* ctx = st->sys->ctx;
  QLB_CUDA_TRY(cudaStreamSynchronize(st->stream));
  int err = 0;
  QLB_CUDA_TRY(cudaMemcpy(&err, st->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    QLB_CUDA_TRY(cudaMemset(st->d_err, 0, sizeof(int)));
    set_error(err & 2 ? "non-finite values met in a truncation" : "a Jacobi eigen-solve hit its sweep limit");
    return err & 2 ? QLB_ENONFINITE : QLB_ENOTCONV;
  }
  return QLB_OK;
}

// ------------------------------------------------------------------ observables

// E[l'][l][0] = delta_{l' l} for l, l' < d[0] (trace over the purification index)
__global__ void k_transfer_start(zd* E, const int* d, long cap) {
  const long mu = d[0];
  for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < mu * mu && x < cap; x += (long)gridDim.x * blockDim.x)
    E[x] = mk<double>((x / mu) == (x % mu) ? 1.0 : 0.0, 0.0);
}

// Builder-layout MPO -> step layout [s'][a][s][b] in new device buffers.
qlb_status mpo_step_layout(qlb_ctx* ctx, const Mpo& Wb, std::vector<zd*>& out, cudaStream_t sm) {
  out.assign(Wb.L, nullptr);
  for (int i = 0; i < Wb.L; i++) {
    long n = (long)Wb.D[i] * 4 * Wb.D[i + 1];
    qlb_status s = dev_alloc(ctx, (void**)&out[i], sizeof(zd) * n);
    if (s) return s;
    k_to_step_layout<<<nblk(n), 256, 0, sm>>>(Wb.core[i], Wb.D[i], Wb.D[i + 1], out[i]);
  }
  QLB_CUDA_TRY(cudaGetLastError());
  return QLB_OK;
}

// Tr(O rho) by the transfer E[l'][l][a] (bra, ket, MPO bond):
//   Y_l'[a][(s,r)] = sum_l E_l'[l][a] A[l][(s,r)]
//   Z[(l',s')][(r,b)] = sum_{a,s} Y_l'[(a,s)][r] W_s'[(a,s)][b]
//   E'[r'][(r,b)] = sum_{(l',s')} conj(A[(l',s')][r']) Z[(l',s')][(r,b)]
// starting from E[mu'][mu][0] = delta (trace over the purification index).  The
// shapes are read from the state's device dims and the buffers belong to the
// state (grown only when the op's MPO bonds need more), so a call allocates
// nothing once the state has seen an op of this size, and it synchronises once,
// for the result.
qlb_status expectation_mpo(qlb_state* st, const std::vector<zd*>& W, const std::vector<int>& D, double* out) {
  qlb_ctx* ctx = st->sys->ctx;
  const int L = st->L;
  const std::vector<int>& hd = st->cap_state;
  auto cap = [&](int i) { return (size_t)hd[SB(i)]; };
  size_t nE = 1, nY = 1, nZ = 1;
  for (int i = 0; i < L; i++) {
    nE = std::max(nE, cap(i) * cap(i) * D[i]);
    nE = std::max(nE, cap(i + 1) * cap(i + 1) * D[i + 1]);
    nY = std::max(nY, cap(i) * D[i] * 2 * cap(i + 1));
    nZ = std::max(nZ, cap(i) * 2 * cap(i + 1) * D[i + 1]);
  }
  qlb_status s;
  {
    size_t a = st->noE, b = st->noE;
    if ((s = realloc_buf(ctx, &st->oE0, &a, nE)) || (s = realloc_buf(ctx, &st->oE1, &b, nE))) return s;
    st->noE = std::max(st->noE, nE);
  }
  if ((s = realloc_buf(ctx, &st->oY, &st->noY, nY)) || (s = realloc_buf(ctx, &st->oZ, &st->noZ, nZ))) return s;
  zd *E0 = st->oE0, *E1 = st->oE1, *Y = st->oY, *Z = st->oZ;
  k_transfer_start<<<nblk((long)cap(0) * cap(0)), 256, 0, st->stream>>>(E0, st->d_dims, (long)nE);
  QLB_CUDA_TRY(cudaGetLastError());
  for (int i = 0; i < L; i++) {
    const int Dl = D[i], Dr = D[i + 1];
    GemmDesc g = gdesc();
    g.A = E0;
    g.B = st->site[i];
    g.C = Y;
    g.m = dconst(Dl);
    g.n = dvar(SB(i + 1), 2);
    g.k = dvar(SB(i));
    g.opA = OP_T;
    g.lda = dconst(Dl);
    g.ldb = dvar(SB(i + 1), 2);
    g.ldc = dvar(SB(i + 1), 2);
    g.sA1 = dvar(SB(i), Dl);
    g.sC1 = dvar(SB(i + 1), 2 * Dl);
    g.nb1 = dvar(SB(i));
    g.m_max = Dl;
    g.n_max = 2 * (int)cap(i + 1);
    g.nb_max = (int)cap(i);
    QLB_CUDA_TRY(launch_gemm<double>(g, st->d_dims, st->stream, nullptr));
    g = gdesc();
    g.A = Y;
    g.B = W[i];
    g.C = Z;
    g.m = dvar(SB(i + 1));
    g.n = dconst(Dr);
    g.k = dconst(2 * Dl);
    g.opA = OP_T;
    g.lda = dvar(SB(i + 1));
    g.ldb = dconst(Dr);
    g.ldc = dconst(Dr);
    g.sA1 = dvar(SB(i + 1), 2 * Dl);
    g.sB2 = dconst(Dl * 2 * Dr);
    g.sC1 = dvar(SB(i + 1), 2 * Dr);
    g.sC2 = dvar(SB(i + 1), Dr);
    g.nb1 = dvar(SB(i));
    g.nb2 = dconst(2);
    g.m_max = (int)cap(i + 1);
    g.n_max = Dr;
    g.nb_max = 2 * (int)cap(i);
    QLB_CUDA_TRY(launch_gemm<double>(g, st->d_dims, st->stream, nullptr));
    g = gdesc();
    g.A = st->site[i];
    g.B = Z;
    g.C = E1;
    g.m = dvar(SB(i + 1));
    g.n = dvar(SB(i + 1), Dr);
    g.k = dvar(SB(i), 2);
    g.opA = OP_C;
    g.lda = dvar(SB(i + 1));
    g.ldb = dvar(SB(i + 1), Dr);
    g.ldc = dvar(SB(i + 1), Dr);
    g.m_max = (int)cap(i + 1);
    g.n_max = (int)cap(i + 1) * Dr;
    QLB_CUDA_TRY(launch_gemm<double>(g, st->d_dims, st->stream, nullptr));
    std::swap(E0, E1);
  }
  zd res;
  QLB_CUDA_TRY(cudaMemcpyAsync(&res, E0, sizeof(zd), cudaMemcpyDeviceToHost, st->stream));
  QLB_CUDA_TRY(cudaStreamSynchronize(st->stream));
  out[0] = res.re;
  out[1] = res.im;
  return QLB_OK;
}

// Branch k of the stacked Kraus MPO (with the drive coefficient of the state's
// current step written in) as a builder-layout MPO with left boundary 1.
qlb_status kraus_branch(qlb_state* st, int k, Mpo& out) {
  qlb_ctx* ctx = st->sys->ctx;
  const Kraus& K = st->kraus;
  if (k < 0 || k >= K.B) {
    set_error("branch index out of range");
    return QLB_EINVAL;
  }
  if (K.driven)
    k_drive_rewrite<<<1, 256, 0, st->stream>>>(K.W[0], K.drive_core0, K.B, K.D[1], K.drive_off, K.drive_D1,
                                                st->sys->d_f, st->sys->n_f, st->d_step, K.dt);
  mpo_clear(ctx, out);
  out.L = K.L;
  out.D = K.D;
  out.D[0] = 1;
  out.core.assign(K.L, nullptr);
  for (int i = 0; i < K.L; i++) {
    long n = (long)out.D[i] * 4 * out.D[i + 1];
    qlb_status s = dev_alloc(ctx, (void**)&out.core[i], sizeof(zd) * n);
    if (s) return s;
    k_from_step_layout<<<nblk(n), 256, 0, st->stream>>>(K.W[i], K.D[i], K.D[i + 1], i == 0 ? k : -1, out.core[i]);
  }
  QLB_CUDA_TRY(cudaGetLastError());
  QLB_CUDA_TRY(cudaStreamSynchronize(st->stream));
  return QLB_OK;
}

// ------------------------------------------------------------------ groups
//
// A group steps S states with one launch per position of the step: each member's
// step is recorded (the same helpers, with every pointer and shape of that
// member), the records are checked to form the same launch sequence, the members'
// descriptors go to one device table, and the grouped launches (blockIdx.y =
// member) are captured once as a CUDA graph on the group's stream.  A member's
// launch computes exactly what its own launch computes: the same kernels, the same
// K split of its GEMMs (decided on the full grid) and the same reduction orders.

void GroupExec::release() {
  if (graph) cudaGraphExecDestroy(graph);
  graph = nullptr;
  if (d_tab) dev_free(ctx, d_tab);
  d_tab = nullptr;
  keys.clear();
  who.clear();
  launches = 0;
}

static size_t rec_row_bytes(int kind) {
  switch (kind) {
    case REC_GEMM:
      return sizeof(GemmDesc);
    case REC_ZIPQR:
    case REC_EIG:
      return sizeof(EigDesc);
    case REC_COPY:
      return sizeof(CopyArgs);
    case REC_BEGIN:
      return sizeof(StepBeginArgs);
    case REC_END:
      return sizeof(StepEndArgs);
    default:
      return 0;  // REC_GEMM_TC: launched member by member
  }
}

static qlb_status group_capture(GroupExec& gx, const std::vector<qlb_state*>& ms, cudaStream_t gs) {
  qlb_ctx* ctx = gx.ctx;
  const int S = (int)ms.size();
  // the previous graph may still run and read the table that is replaced below
  QLB_CUDA_TRY(cudaStreamSynchronize(gs));
  std::vector<std::vector<LaunchRec>> recs(S);
  for (int pass = 0; pass < 2; pass++) {
    for (int m = 0; m < S; m++) {
      recs[m].clear();
      ms[m]->rec = &recs[m];
      qlb_status s = enqueue_step(ms[m], ms[m]->kraus, true);
      ms[m]->rec = nullptr;
      if (s) return s;
    }
    if (pass == 1) break;
    // an eigen-solve served by the kernel of a larger co-member may need more
    // workspace than the member's own plan gave it: grow it, then record again
    // (the records hold the workspace pointers)
    bool grown = false;
    for (size_t p = 0; p < recs[0].size(); p++) {
      if (recs[0][p].kind != REC_EIG) continue;
      int gmax = 1;
      for (int m = 0; m < S; m++)
        if (p < recs[m].size()) gmax = std::max(gmax, recs[m][p].e.n_max);
      for (int m = 0; m < S; m++) {
        if (p >= recs[m].size()) continue;
        const size_t need = eig_group_workspace_elems(recs[m][p].e.n_max, gmax);
        if (need > ms[m]->nEw) {
          qlb_status s = realloc_buf(ctx, &ms[m]->eigw, &ms[m]->nEw, need);
          if (s) return s;
          ms[m]->plan_key++;  // the member's own captured step used the old workspace
          grown = true;
        }
      }
    }
    if (!grown) break;
  }
  const size_t P = recs[0].size();
  for (int m = 1; m < S; m++) {
    bool same = recs[m].size() == P;
    for (size_t p = 0; same && p < P; p++)
      same = recs[m][p].kind == recs[0][p].kind && recs[m][p].df == recs[0][p].df;
    if (!same) {
      set_error("the states of a group must step the same launch sequence (same sites, precision form and scheme)");
      return QLB_EINVAL;
    }
  }
  for (size_t p = 0; p < P; p++)
    if (recs[0][p].kind == REC_GEMM)
      for (int m = 0; m < S; m++)
        if (!recs[m][p].g.ws) {
          set_error("group GEMM without a workspace");
          return QLB_EINVAL;
        }
  // the table: for each position, S rows of its argument type, 16-byte aligned
  std::vector<size_t> off(P, 0);
  size_t total = 0;
  for (size_t p = 0; p < P; p++) {
    off[p] = total;
    total += ((size_t)S * rec_row_bytes(recs[0][p].kind) + 15) & ~(size_t)15;
  }
  std::vector<unsigned char> host(std::max<size_t>(total, 16));
  for (size_t p = 0; p < P; p++) {
    const size_t rb = rec_row_bytes(recs[0][p].kind);
    for (int m = 0; m < S && rb; m++) {
      const LaunchRec& r = recs[m][p];
      const void* src = nullptr;
      switch (r.kind) {
        case REC_GEMM: src = &r.g; break;
        case REC_ZIPQR:
        case REC_EIG: src = &r.e; break;
        case REC_COPY: src = &r.c; break;
        case REC_BEGIN: src = &r.b; break;
        case REC_END: src = &r.x; break;
      }
      std::memcpy(host.data() + off[p] + (size_t)m * rb, src, rb);
    }
  }
  gx.release();
  qlb_status s;
  if ((s = dev_alloc(ctx, &gx.d_tab, host.size()))) return s;
  QLB_CUDA_TRY(cudaMemcpyAsync(gx.d_tab, host.data(), host.size(), cudaMemcpyHostToDevice, gs));
  QLB_CUDA_TRY(cudaStreamSynchronize(gs));
  unsigned char* tab = (unsigned char*)gx.d_tab;
  QLB_CUDA_TRY(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  int launches = 0;
  for (size_t p = 0; p < P && e == cudaSuccess; p++) {
    const LaunchRec& r0 = recs[0][p];
    unsigned char* t = tab + off[p];
    long maxn = 1;
    int n_max = 1;
    for (int m = 0; m < S; m++) {
      maxn = std::max(maxn, recs[m][p].grid_n);
      n_max = std::max(n_max, recs[m][p].e.n_max);
    }
    launches++;
    switch (r0.kind) {
      case REC_BEGIN:
        k_step_begin_grp<<<dim3(nblk(maxn), S), 256, 0, gs>>>((const StepBeginArgs*)t);
        e = cudaGetLastError();
        break;
      case REC_END:
        k_step_end_grp<<<dim3(1, S), 32, 0, gs>>>((const StepEndArgs*)t);
        e = cudaGetLastError();
        break;
      case REC_COPY:
        k_copy_grp<<<dim3(nblk(maxn), S), 256, 0, gs>>>((const CopyArgs*)t);
        e = cudaGetLastError();
        break;
      case REC_GEMM:
        e = launch_gemm_group((const GemmDesc*)t, S, r0.df, gs, nullptr);
        break;
      case REC_GEMM_TC:
        launches += S - 1;
        for (int m = 0; m < S && e == cudaSuccess; m++)
          e = launch_gemm_tc(recs[m][p].g, recs[m][p].dims, gs, recs[m][p].err, nullptr);
        break;
      case REC_ZIPQR:
        e = r0.df ? launch_zipqr_group<df64>(n_max, (const EigDesc*)t, S, gs, nullptr)
                  : launch_zipqr_group<double>(n_max, (const EigDesc*)t, S, gs, nullptr);
        break;
      case REC_EIG:
        e = r0.df ? launch_eig_group<df64>(n_max, (const EigDesc*)t, S, gs, nullptr)
                  : launch_eig_group<double>(n_max, (const EigDesc*)t, S, gs, nullptr);
        break;
    }
  }
  cudaGraph_t gr = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(gs, &gr);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    set_error(std::string("group capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    return QLB_EDEVICE;
  }
  e = cudaGraphInstantiate(&gx.graph, gr, 0);
  cudaGraphDestroy(gr);
  QLB_CUDA_TRY(e);
  gx.keys.resize(S);
  gx.who.resize(S);
  for (int m = 0; m < S; m++) gx.who[m] = ms[m]->uid;
  for (int m = 0; m < S; m++) gx.keys[m] = ms[m]->plan_key;
  gx.launches = launches;
  return QLB_OK;
}

qlb_status group_run(GroupExec& gx, const std::vector<qlb_state*>& ms, cudaStream_t gs, cudaEvent_t ev, int64_t n,
                     bool sync) {
  if (n <= 0 || ms.empty()) return QLB_OK;
  bool fresh = gx.graph && gx.keys.size() == ms.size() && gx.who.size() == ms.size();
  for (size_t m = 0; fresh && m < ms.size(); m++) fresh = gx.who[m] == ms[m]->uid && gx.keys[m] == ms[m]->plan_key;
  qlb_status s;
  // the members' earlier work (their own streams) comes first
  for (qlb_state* st : ms) {
    QLB_CUDA_TRY(cudaEventRecord(ev, st->stream));
    QLB_CUDA_TRY(cudaStreamWaitEvent(gs, ev, 0));
  }
  if (!fresh && (s = group_capture(gx, ms, gs))) return s;
  for (int64_t k = 0; k < n; k++) QLB_CUDA_TRY(cudaGraphLaunch(gx.graph, gs));
  // and their later work waits for the group's steps
  QLB_CUDA_TRY(cudaEventRecord(ev, gs));
  for (qlb_state* st : ms) {
    QLB_CUDA_TRY(cudaStreamWaitEvent(st->stream, ev, 0));
    st->host_steps += n;
  }
  if (!sync) return QLB_OK;
  QLB_CUDA_TRY(cudaStreamSynchronize(gs));
  for (qlb_state* st : ms)
    if ((s = check_flags(st))) return s;
  return QLB_OK;
}

qlb_status state_sum_abs2_site0(qlb_state* st, double* out) {
  qlb_ctx* ctx = st->sys->ctx;
  double* d = st->d_stats + 3;
  k_sum_abs2<<<1, 256, 0, st->stream>>>(st->site[0], dvar2(SB(0), SB(1), 2), st->d_dims, d);
  QLB_CUDA_TRY(cudaMemcpyAsync(out, d, sizeof(double), cudaMemcpyDeviceToHost, st->stream));
  QLB_CUDA_TRY(cudaStreamSynchronize(st->stream));
  return QLB_OK;
}

}  // namespace qlb
