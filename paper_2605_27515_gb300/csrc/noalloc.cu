// qlb_purity_noalloc: purity of a state without any device allocation.
//
// qlb_purity allocates a small Gram buffer and an accumulator on every call.
// This variant runs the same Gram GEMM and reduction in a fixed scratch array that
// lives in the library's own device image (a file-scope __device__ array), so it
// never calls cudaMalloc or cudaFree.  That matters for callers that may not
// allocate at that moment: callers whose device memory is owned by another
// allocator with a fixed budget, and latency-sensitive monitoring loops that
// cannot afford the device-wide synchronisation that cudaFree implies.  The call
// itself synchronises (it reads the bond dimensions back and waits for the
// result), so it is not meant for use inside CUDA stream capture.

#include <mutex>

#include "step.cuh"

#define QLB_API extern "C" __attribute__((visibility("default")))

namespace qlb {
namespace {

// Largest purification rank the scratch array serves.
constexpr int NOALLOC_MAX_MU = 128;

}  // namespace
}  // namespace qlb

// Gram matrix (NOALLOC_MAX_MU^2 complex doubles) followed by two result slots.
// Every GPU that loads the library holds this array (about 256 KB) until exit.
// In host code this name is only a host-side stand-in: kernels get the device
// address looked up by cudaGetSymbolAddress below.
static __device__ __align__(256) double g_purity_scratch[2 * qlb::NOALLOC_MAX_MU * qlb::NOALLOC_MAX_MU + 8];

namespace qlb {
namespace {

// out2[0] = sum |G|^2 over the mu x mu Gram, out2[1] = sum |A_0|^2.  One CTA, the
// results are written (not accumulated), so the stale contents of a previous
// call never leak into this one.
__global__ void k_purity_reduce(const zd* G, int mu, const zd* A0, long nA0, double* out2) {
  __shared__ double sh[2][32];
  double g = 0, a = 0;
  for (long x = threadIdx.x; x < (long)mu * mu; x += blockDim.x) g += cabs2(G[x]);
  for (long x = threadIdx.x; x < nA0; x += blockDim.x) a += cabs2(A0[x]);
  for (int o = 16; o > 0; o >>= 1) {
    g += __shfl_xor_sync(0xffffffffu, g, o);
    a += __shfl_xor_sync(0xffffffffu, a, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = g;
    sh[1][threadIdx.x >> 5] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double rg = 0, ra = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      rg += sh[0][w];
      ra += sh[1][w];
    }
    out2[0] = rg;
    out2[1] = ra;
  }
}

std::mutex g_scratch_mutex;
constexpr int MAX_DEVICES = 64;
double* g_scratch_addr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device, looked up once per
// device with that device current.
qlb_status scratch_address(int device, double** out) {
  if (device < 0 || device >= MAX_DEVICES) {
    set_error("device ordinal out of range for the no-alloc scratch");
    return QLB_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_purity_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress(g_purity_scratch): ") + cudaGetErrorString(e));
      return QLB_EDEVICE;
    }
    g_scratch_addr[device] = (double*)p;
  }
  *out = g_scratch_addr[device];
  return QLB_OK;
}

}  // namespace
}  // namespace qlb

using namespace qlb;

QLB_API qlb_status qlb_purity_noalloc(qlb_state* st, double* out) {
  if (!st || !out) {
    set_error("null argument");
    return QLB_EINVAL;
  }
  qlb_ctx* ctx = st->sys->ctx;
  int prev = -1;
  QLB_CUDA_TRY(cudaGetDevice(&prev));
  if (prev != ctx->opt.device) QLB_CUDA_TRY(cudaSetDevice(ctx->opt.device));
  struct Restore {
    int dev, prev;
    ~Restore() {
      if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
  } restore{ctx->opt.device, prev};
  std::vector<int> d;
  qlb_status s;
  if ((s = read_dims(st, d))) return s;
  const int mu = d[0], r = d[1];
  if (mu < 1 || mu > NOALLOC_MAX_MU) {
    set_error("qlb_purity_noalloc serves purification ranks up to " + std::to_string(NOALLOC_MAX_MU) +
              "; this state has " + std::to_string(mu));
    return QLB_EINVAL;
  }
  double* scratch = nullptr;
  if ((s = scratch_address(ctx->opt.device, &scratch))) return s;
  zd* G = (zd*)scratch;
  double* res = scratch + 2 * NOALLOC_MAX_MU * NOALLOC_MAX_MU;
  // G = A_0 A_0^dag (mu x mu), the same GEMM as qlb_purity
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
  k_purity_reduce<<<1, 256, 0, st->stream>>>(G, mu, st->site[0], (long)mu * 2 * r, res);
  QLB_CUDA_TRY(cudaGetLastError());
  double h[2] = {0, 0};
  QLB_CUDA_TRY(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st->stream));
  QLB_CUDA_TRY(cudaStreamSynchronize(st->stream));
  *out = h[1] > 0 ? h[0] / (h[1] * h[1]) : 0.0;
  return QLB_OK;
}
