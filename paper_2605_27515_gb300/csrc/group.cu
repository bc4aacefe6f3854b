// Groups of states stepped with one launch per phase of the step (include/qlb.h,
// "groups").  The recording, the device table of member descriptors and the
// captured graph are in step.cu (group_run); this file holds the handle and its
// argument checks.

#include <algorithm>
#include <cmath>
#include <set>
#include <vector>

#include "step.cuh"

#define QLB_API extern "C" __attribute__((visibility("default")))

using namespace qlb;

struct qlb_group {
  qlb_ctx* ctx = nullptr;
  std::vector<qlb_state*> members;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  GroupExec exec;
};

#define CHECK_ARG(cond, msg) \
  do {                       \
    if (!(cond)) {           \
      set_error(msg);        \
      return QLB_EINVAL;     \
    }                        \
  } while (0)

QLB_API qlb_status qlb_group_create(qlb_ctx* ctx, qlb_state* const* states, int n_states, qlb_group** out) {
  CHECK_ARG(ctx && states && out, "null argument");
  *out = nullptr;
  CHECK_ARG(n_states >= 1 && n_states <= 4096, "n_states must be in 1..4096");
  std::set<qlb_state*> seen;
  for (int m = 0; m < n_states; m++) {
    qlb_state* st = states[m];
    CHECK_ARG(st, "null state in the group");
    CHECK_ARG(st->sys && st->sys->ctx == ctx, "every state of a group must belong to the group's context");
    CHECK_ARG(seen.insert(st).second, "a state appears twice in the group");
    CHECK_ARG(st->L == states[0]->L, "the states of a group must have the same number of sites");
    CHECK_ARG(st->prec == states[0]->prec, "the states of a group must use the same precision form");
    CHECK_ARG(st->sys->order == states[0]->sys->order, "the states of a group must use the same Kraus scheme");
  }
  QLB_CUDA_TRY(cudaSetDevice(ctx->opt.device));
  qlb_group* g = new qlb_group();
  g->ctx = ctx;
  g->members.assign(states, states + n_states);
  g->exec.ctx = ctx;
  if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming) != cudaSuccess) {
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
    set_error("group stream or event creation failed");
    return QLB_EDEVICE;
  }
  *out = g;
  return QLB_OK;
}

QLB_API void qlb_group_destroy(qlb_group* g) {
  if (!g) return;
  cudaStreamSynchronize(g->stream);
  g->exec.release();
  cudaEventDestroy(g->ev);
  cudaStreamDestroy(g->stream);
  delete g;
}

QLB_API qlb_status qlb_group_step(qlb_group* g, double dt, int64_t n) {
  CHECK_ARG(g, "null group");
  CHECK_ARG(std::isfinite(dt) && dt > 0, "dt must be positive and finite");
  CHECK_ARG(n >= 0, "n must be >= 0");
  qlb_status s;
  bool unstable = false;
  // every member's Kraus MPO for dt and its buffers, as qlb_step plans them
  for (qlb_state* st : g->members) {
    CHECK_ARG(st->sys->order == g->members[0]->sys->order, "a member's Kraus scheme changed since the group was made");
    bool rebuilt = !(st->kraus.dt == dt && st->kraus.version == st->sys->version);
    if ((s = build_kraus(st, dt))) return s;
    if (rebuilt && (s = plan_buffers(st, st->kraus))) return s;
    unstable = unstable || st->kraus.unstable_factor > 4.0;
  }
  if ((s = group_run(g->exec, g->members, g->stream, g->ev, n, !g->ctx->opt.stream_ordered))) return s;
  return unstable ? QLB_WUNSTABLE : QLB_OK;
}

QLB_API qlb_status qlb_group_launches(qlb_group* g, int* per_step) {
  CHECK_ARG(g && per_step, "null argument");
  *per_step = g->exec.launches;
  return QLB_OK;
}

QLB_API qlb_status qlb_group_stream(qlb_group* g, void** stream) {
  CHECK_ARG(g && stream, "null argument");
  *stream = (void*)g->stream;
  return QLB_OK;
}
