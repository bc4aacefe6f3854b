// Autotuner of the launch shapes of the step: the cap on the run-time K split of
// the zip-up Gram GEMM G = M M^dag, whose (2z) x (2z) output makes few 32 x 32 tiles
// over a long K = d D (the work-distributed GEMM splits K until its fixed grid is
// full; more parts mean more partial tiles to add).  For every bucket (rows m,
// inner size K) the tuner times the GEMM with caps 1, 2, 4, 8, 16 with CUDA events
// (best of three, on random data in a scratch allocation) and keeps the fastest;
// the table lives in the context and can be written to / read from a text file of
// lines "m K ksplit", so a tuning run on one GPU serves later runs.

#include <algorithm>
#include <cstdio>
#include <random>
#include <vector>

#include "builder.cuh"

#define QLB_API extern "C" __attribute__((visibility("default")))

namespace qlb {

namespace {

const int kTuneM[] = {32, 64, 128, 256};
const int kTuneK[] = {256, 1024, 4096};
const int kTuneSplit[] = {1, 2, 4, 8, 16};

int bucket_m(long m) {
  for (int b : kTuneM)
    if (m <= b) return b;
  return kTuneM[3];
}
int bucket_k(long K) {
  for (int b : kTuneK)
    if (K <= b) return b;
  return kTuneK[2];
}

}  // namespace

int gram_splitk(const qlb_ctx* ctx, long mm, long kk) {
  if (ctx && !ctx->gram_tune.empty()) {
    auto it = ctx->gram_tune.find({bucket_m(mm), bucket_k(kk)});
    if (it != ctx->gram_tune.end()) return std::max(1, std::min(it->second, (int)std::max<long>(1, kk / 16)));
  }
  return 0;  // no cap: the kernel's own run-time rule
}

}  // namespace qlb

using namespace qlb;

QLB_API qlb_status qlb_autotune(qlb_ctx* ctx, const char* path) {
  if (!ctx) {
    set_error("null context");
    return QLB_EINVAL;
  }
  QLB_CUDA_TRY(cudaSetDevice(ctx->opt.device));
  const long mmax = kTuneM[3], kmax = kTuneK[2];
  zd *M = nullptr, *G = nullptr, *W = nullptr;
  auto cleanup = [&]() {
    cudaFree(M);
    cudaFree(G);
    cudaFree(W);
  };
  if (cudaMalloc(&M, sizeof(zd) * mmax * kmax) != cudaSuccess || cudaMalloc(&G, sizeof(zd) * mmax * mmax) != cudaSuccess ||
      cudaMalloc(&W, sizeof(zd) * gemm_workspace_elems(gemm_grid_default())) != cudaSuccess ||
      cudaMemset(W, 0, sizeof(zd) * gemm_workspace_elems(gemm_grid_default())) != cudaSuccess) {
    cleanup();
    set_error("qlb_autotune: scratch allocation failed");
    return QLB_ENOMEM;
  }
  {
    std::vector<zd> h(mmax * kmax);
    std::mt19937_64 rng(12345);
    std::normal_distribution<double> nd;
    for (auto& z : h) z = mk<double>(nd(rng), nd(rng));
    cudaMemcpy(M, h.data(), sizeof(zd) * h.size(), cudaMemcpyHostToDevice);
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  std::map<std::pair<int, int>, int> table;
  qlb_status st = QLB_OK;
  for (int m : kTuneM)
    for (int K : kTuneK) {
      float best = 1e30f;
      int best_ks = 1;
      for (int ks : kTuneSplit) {
        GemmDesc g{};
        g.A = M;
        g.B = M;
        g.C = G;
        g.m = g.n = dconst(m);
        g.k = dconst(K);
        g.opB = OP_C;
        g.lda = g.ldb = dconst(K);
        g.ldc = dconst(m);
        g.sA1 = g.sB1 = g.sC1 = g.sA2 = g.sB2 = g.sC2 = dconst(0);
        g.nb1 = g.nb2 = dconst(1);
        g.alpha_re = 1.0;
        g.m_max = g.n_max = m;
        g.nb_max = 1;
        g.ksplit = ks;
        g.ws = W;
        float t = 1e30f;
        for (int rep = 0; rep < 4; rep++) {
          cudaEventRecord(a, 0);
          cudaError_t e = launch_gemm<double>(g, nullptr, 0, nullptr);
          cudaEventRecord(b, 0);
          if (e == cudaSuccess) e = cudaEventSynchronize(b);
          if (e != cudaSuccess) {
            set_error(std::string("qlb_autotune: ") + cudaGetErrorString(e));
            st = QLB_EDEVICE;
            break;
          }
          float ms = 0;
          cudaEventElapsedTime(&ms, a, b);
          if (rep > 0) t = std::min(t, ms);  // the first launch warms up
        }
        if (st) break;
        if (t < best) {
          best = t;
          best_ks = ks;
        }
      }
      if (st) break;
      table[{m, K}] = best_ks;
    }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cleanup();
  if (st) return st;
  ctx->gram_tune = table;
  if (path && *path) {
    FILE* f = fopen(path, "w");
    if (!f) {
      set_error(std::string("qlb_autotune: cannot write ") + path);
      return QLB_EINVAL;
    }
    fprintf(f, "# m K ksplit  (split-K of the Gram GEMM, fastest of 1 2 4 8 16 by CUDA events)\n");
    for (auto& kv : table) fprintf(f, "%d %d %d\n", kv.first.first, kv.first.second, kv.second);
    fclose(f);
  }
  return QLB_OK;
}

QLB_API qlb_status qlb_load_tuning(qlb_ctx* ctx, const char* path) {
  if (!ctx || !path) {
    set_error("null argument");
    return QLB_EINVAL;
  }
  FILE* f = fopen(path, "r");
  if (!f) {
    set_error(std::string("qlb_load_tuning: cannot read ") + path);
    return QLB_EINVAL;
  }
  std::map<std::pair<int, int>, int> table;
  char line[256];
  while (fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    int m, K, ks;
    if (sscanf(line, "%d %d %d", &m, &K, &ks) == 3 && m > 0 && K > 0 && ks >= 1 && ks <= 64) table[{m, K}] = ks;
  }
  fclose(f);
  if (table.empty()) {
    set_error(std::string("qlb_load_tuning: no entries in ") + path);
    return QLB_EINVAL;
  }
  ctx->gram_tune = table;
  return QLB_OK;
}
