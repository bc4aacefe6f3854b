// Object model behind the opaque C-ABI handles.
#pragma once

#include <atomic>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "qlb_internal.cuh"

namespace qlb {

struct Kraus;

// ------------------------------------------------------------------ device buffers

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// ------------------------------------------------------------------ MPOs
//
// Builder layout: core i is W[a][p][b] with p = 2*s_out + s_in (the TT-SVD order of
// the dense matrix).  Step layout: W[s_out][a][s_in][b].
struct Mpo {
  int L = 0;
  std::vector<int> D;      // D[0..L]; D[0] = left boundary (1, or B branches), D[L] = 1
  std::vector<zd*> core;   // device pointers, builder layout
  ~Mpo();
  Mpo() = default;
  Mpo(const Mpo&) = delete;
  Mpo& operator=(const Mpo&) = delete;
  size_t bytes() const;
};

// A term of an operator, kept on the device: coeff * (x)_m F_m (F_m null = identity).
struct DevTerm {
  zd coeff;
  std::vector<zd*> fac;  // one per mode; owned by the op (shared_ptr-free: freed with the op)
  // per mode, a recipe naming the factor when it is made of built-in factors only
  // ("" for caller matrices); equal recipes on equal R give equal matrices, so
  // their MPOs are cached by the context
  std::vector<std::string> key;
};

}  // namespace qlb

struct qlb_ctx {
  qlb_options opt;
  cudaStream_t stream = nullptr;
  size_t mem_held = 0;
  long long n_allocs = 0;  // device allocations made for this context so far
  // eigen-solver counters, updated by every solve of the context's states (also
  // inside captured graphs): [0] solves, [1] Jacobi sweeps / QL passes, [2] sum of
  // runtime sizes n, [3] sum of kept counts k, [4] solves that hit the sweep limit
  double* d_solver = nullptr;
  // profiling
  bool prof_on = false;
  struct PEv {
    int kclass;
    cudaEvent_t a, b;
  };
  std::vector<PEv> prof_events;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  double* d_prof = nullptr;  // [QLB_K_COUNT] flops, [QLB_K_COUNT..2*] bytes
  double prof_ms[QLB_K_COUNT] = {0};
  long long prof_launch[QLB_K_COUNT] = {0};
  // split-K factor of the Gram GEMM per (rows bucket, K bucket), from the autotuner
  // (qlb_autotune) or a table it wrote (qlb_load_tuning); empty: the built-in rule
  std::map<std::pair<int, int>, int> gram_tune;
  // MPOs of built-in per-mode factors, keyed by "R|recipe" (see DevTerm::key)
  std::map<std::string, qlb::Mpo*> factor_mpo_cache;
  ~qlb_ctx();
};

struct qlb_system {
  qlb_ctx* ctx = nullptr;
  int M = 0;
  std::vector<int> R;
  int L = 0;
  const qlb_op* H0 = nullptr;
  const qlb_op* H1 = nullptr;
  std::vector<double> f_table;
  double* d_f = nullptr;
  int64_t n_f = 0;
  std::vector<const qlb_op*> jumps;
  int version = 0;  // bumped when H or jumps change
  int order = 1;    // Kraus scheme order (1 or 2)
  // Kraus MPO of the last (dt, version) built by any state of this system; new
  // states copy it instead of rebuilding (owned, freed with the system)
  qlb::Kraus* kraus_tmpl = nullptr;
  ~qlb_system();
};

struct qlb_op {
  qlb_system* sys = nullptr;
  std::vector<qlb::DevTerm> terms;
  std::vector<qlb::zd*> owned;  // device dense factors owned by this op
  qlb::Mpo mpo;
  std::vector<qlb::zd*> step_core;  // the MPO in step layout, made on first use by qlb_expectation
  double inf_norm_bound = 0.0;  // sum_t |c_t| prod_m ||F_m||_inf
  ~qlb_op();
};

namespace qlb {

// Stacked Kraus MPO of one step (Sec. V.B): branch k on the left boundary.
struct Kraus {
  double dt = -1;
  int version = -1;
  int B = 0;            // branches = 1 + number of jumps
  int L = 0;
  std::vector<int> D;   // D[0] = B
  std::vector<zd*> W;   // step layout [s'][a][s][b]
  bool driven = false;
  int drive_off = 0;    // first column of the H1 block in bond 1
  int drive_D1 = 0;     // its width
  zd* drive_core0 = nullptr;  // H1 core 0, builder layout [1][4][drive_D1], unscaled
  double unstable_factor = 0;  // h * gamma_bound
  ~Kraus();
};

// Arguments of the small launches of a step (also the rows of a group's table).
struct StepBeginArgs {
  int* d;
  int L, B;
  zd* C0;
  long c0_cap;
  zd* W0;
  const zd* h1c0;
  int D1tot, drive_off, drive_D1;
  const double* f;
  long long n_f;
  const long long* step;
  double dt;
  double* stats;
};
struct StepEndArgs {
  long long* step;
  int count;
};
struct CopyArgs {
  zd* dst;
  const zd* src;
  DimExpr cnt;
  const int* d;
};

// One launch of a step as recorded (instead of launched) when the state steps as
// a member of a group: the group launches each position of its members' records
// once, over all members.
enum RecKind { REC_BEGIN = 0, REC_END, REC_GEMM, REC_GEMM_TC, REC_ZIPQR, REC_EIG, REC_COPY };
struct LaunchRec {
  int kind = 0;
  int df = 0;        // ZIPQR / EIG: double-float (mixed forms); GEMM: the df64 flag
  int kclass = 0;    // profiling class
  long grid_n = 0;   // BEGIN / COPY: elements the launch covers at most
  GemmDesc g{};
  EigDesc e{};
  CopyArgs c{};
  StepBeginArgs b{};
  StepEndArgs x{};
  int* err = nullptr;  // GEMM_TC: the member's error flags
  const int* dims = nullptr;
};

// A number no other state of the process has had (group graphs are keyed by it:
// a new state may reuse a destroyed one's address).
inline unsigned long long next_state_uid() {
  static std::atomic<unsigned long long> n{0};
  return ++n;
}

}  // namespace qlb

struct qlb_state {
  const unsigned long long uid = qlb::next_state_uid();
  qlb_system* sys = nullptr;
  int L = 0;
  int prec = QLB_PREC_F64;
  // truncation parameters
  double tol = 1e-12;
  int chi_max = 64, chi_mu_max = 16;
  int cap_chi = 64, cap_mu = 16;  // allocation caps
  // every launch that touches this state goes to its own stream, so independent
  // states step concurrently on the GPU; setup work stays on the context stream
  cudaStream_t stream = nullptr;
  // device dims: [0..L] state bonds, [L+1 .. 2L+1] zip-up bonds
  int* d_dims = nullptr;
  std::vector<int> cap_state;  // host capacities of state bonds [0..L]
  // sites (FP64 storage)
  std::vector<qlb::zd*> site;
  std::vector<size_t> site_cap;  // elements
  // scratch
  qlb::zd *X = nullptr, *Mb = nullptr, *G = nullptr, *Cin = nullptr, *Cout = nullptr;
  qlb::zd *T1 = nullptr, *T2 = nullptr, *T3 = nullptr, *eigw = nullptr;
  size_t nX = 0, nM = 0, nG = 0, nC = 0, nT = 0, nEw = 0;
  // transfer-sweep buffers of the observables (grown on demand, reused by later calls)
  qlb::zd *oE0 = nullptr, *oE1 = nullptr, *oY = nullptr, *oZ = nullptr;
  size_t noE = 0, noY = 0, noZ = 0;
  // split-K of the zip-up Gram GEMMs (per site) and their partial-sum workspace
  std::vector<int> gram_split;
  qlb::zd* Wsk = nullptr;
  size_t nWsk = 0;
  double* d_lam = nullptr;
  int* d_gate = nullptr;  // zip-up range basis -> Jacobi solve behind it (1: run)
  double* d_stats = nullptr;  // [0] kept weight (mu), [1] total weight (mu), [2] max disc, [3] scratch
  int* d_err = nullptr;
  long long* d_step = nullptr;  // steps taken (drive table index)
  long long host_steps = 0;
  // planned step
  qlb::Kraus kraus;     // stacked Kraus MPO of the current dt
  qlb::Kraus kraus_id;  // identity (truncate-only passes)
  int plan_key = 0;     // bumped whenever buffers, caps or the Kraus MPO change
  cudaGraphExec_t graph = nullptr;
  int graph_key = -1;
  // set while the state's step is recorded for a group (launches go here instead)
  std::vector<qlb::LaunchRec>* rec = nullptr;
  std::vector<qlb::DevBuf> extra;  // other owned buffers
  ~qlb_state();
};
