// Step planning and enqueueing (internal).
#pragma once

#include "builder.cuh"

namespace qlb {

inline int SB(int i) { return i; }                 // state bond i (0..L)
inline int ZB(const qlb_state* st, int i) { return st->L + 1 + i; }  // zip-up bond i (0..L)

// Builds (or reuses) the stacked Kraus MPO of the system for time step dt.
qlb_status build_kraus(qlb_state* st, double dt);
// The identity "Kraus" MPO (one branch, bond 1) used by truncate-only passes.
qlb_status build_identity_kraus(qlb_state* st);
// Sizes every buffer of the state for its current Kraus MPO and caps.
qlb_status plan_buffers(qlb_state* st, const Kraus& K);
// Enqueues one full step (apply + stack + recompress + purify + renormalise).
qlb_status enqueue_step(qlb_state* st, const Kraus& K, bool count_step);
// One recompression pass with the identity Kraus MPO (truncate / init).
qlb_status truncate_pass(qlb_state* st);
// Sum |A_0|^2 (= Tr rho for a right-canonical state).
qlb_status state_sum_abs2_site0(qlb_state* st, double* out);
// Runs n steps (CUDA graph unless profiling) and checks the device error flags.
qlb_status run_steps(qlb_state* st, int64_t n, bool sync);
// The state's device error flags and trace, read after its work has completed.
qlb_status check_flags(qlb_state* st);

// The captured step of a group of states (one launch per position over all members).
struct GroupExec {
  qlb_ctx* ctx = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::vector<int> keys;   // members' plan keys at capture
  std::vector<unsigned long long> who;  // the members' uids at capture
  void* d_tab = nullptr;   // device table of the members' launch descriptors
  int launches = 0;        // kernel launches per captured step
  void release();
};
// Steps the members n times on stream gs (ordered after, and before, the work of
// their own streams through ev); re-records and re-captures when a member's plan
// changed.  Each member's Kraus MPO and buffers must be planned for the step.
qlb_status group_run(GroupExec& gx, const std::vector<qlb_state*>& ms, cudaStream_t gs, cudaEvent_t ev, int64_t n,
                     bool sync);
// Host copy of the state bonds.
qlb_status read_dims(qlb_state* st, std::vector<int>& d);
// Branch k of the current Kraus MPO as a builder-layout MPO (left boundary 1).
qlb_status kraus_branch(qlb_state* st, int k, Mpo& out);
// Builder-layout MPO -> step-layout cores in new device buffers (launched on sm).
qlb_status mpo_step_layout(qlb_ctx* ctx, const Mpo& W, std::vector<zd*>& out, cudaStream_t sm);
// Tr(O rho) with an MPO in step layout (left boundary 1, bonds D[0..L]).
qlb_status expectation_mpo(qlb_state* st, const std::vector<zd*>& W, const std::vector<int>& D, double* out);

}  // namespace qlb
