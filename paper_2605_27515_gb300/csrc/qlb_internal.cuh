// Internal types of libqlb: complex arithmetic, device-side shape expressions,
// launch descriptors and error plumbing.  Not part of the C-ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "qlb.h"

namespace qlb {

// ------------------------------------------------------------------ complex

template <typename R>
struct cx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) {
  cx<R> z;
  z.re = a;
  z.im = b;
  return z;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) {
  return mk<R>(a.re + b.re, a.im + b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) {
  return mk<R>(a.re - b.re, a.im - b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> cconj(cx<R> a) {
  return mk<R>(a.re, -a.im);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> cscale(cx<R> a, R s) {
  return mk<R>(a.re * s, a.im * s);
}
// acc += a * b
template <typename R>
__host__ __device__ __forceinline__ void cfma(cx<R>& acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
template <typename R>
__host__ __device__ __forceinline__ R cabs2(cx<R> a) {
  return a.re * a.re + a.im * a.im;
}

typedef cx<double> zd;
typedef cx<float> zf;

// ------------------------------------------------------------------ device-side shapes
//
// Bond dimensions change at every truncation and live in device memory, so the
// launches of a step never wait for the host.  A size is written as
//   c * d[a] * d[b]      (a or b < 0 means the factor 1)
// and evaluated inside the kernel from the context's dims array.

struct DimExpr {
  int c, a, b;
};
__host__ __device__ __forceinline__ DimExpr dconst(int c) { return DimExpr{c, -1, -1}; }
__host__ __device__ __forceinline__ DimExpr dvar(int idx, int c = 1) { return DimExpr{c, idx, -1}; }
__host__ __device__ __forceinline__ DimExpr dvar2(int i1, int i2, int c = 1) { return DimExpr{c, i1, i2}; }

__device__ __forceinline__ int dev_eval(const DimExpr& e, const int* d) {
  long v = e.c;
  if (e.a >= 0) v *= d[e.a];
  if (e.b >= 0) v *= d[e.b];
  return (int)v;
}
// Host-side evaluation with a host mirror of the dims (used for capacity bounds).
inline long host_eval(const DimExpr& e, const std::vector<int>& d) {
  long v = e.c;
  if (e.a >= 0) v *= d[e.a];
  if (e.b >= 0) v *= d[e.b];
  return v;
}

// ------------------------------------------------------------------ launch descriptors

enum Op { OP_N = 0, OP_T = 1, OP_C = 2 };

// Batched complex GEMM:  C[b1,b2] = alpha * op(A[b1,b2]) * op(B[b1,b2]) (+ C if beta)
// row-major; op(A) is m x k, op(B) is k x n.  Batch offsets are b1*s?1 + b2*s?2.
struct GemmDesc {
  const void* A;
  const void* B;
  void* C;
  DimExpr m, n, k;
  DimExpr lda, ldb, ldc;
  DimExpr sA1, sB1, sC1, sA2, sB2, sC2;
  DimExpr nb1, nb2;
  int opA, opB;
  double alpha_re, alpha_im;
  const double* alpha_scale;  // optional device scalar multiplying alpha (real)
  int alpha_scale_rsqrt;      // 1: multiply by 1/sqrt(*alpha_scale) instead
  int beta;                   // 1: accumulate into C
  // caps on the grid (host-known maxima)
  int m_max, n_max, nb_max;
  int kclass;  // profiling class
  // Work distribution.  Without ws: one CTA per planned output tile.  With ws (at
  // least gemm_workspace_elems(grid) complex elements, zeroed once): a fixed grid of
  // `grid` CTAs (0 = two per SM) that splits the K range at run time so that tiles x
  // parts fill it; ksplit >= 1 caps that split (0: the default cap).  The last CTA of a tile adds the
  // partials in part order (deterministic).
  int ksplit;
  void* ws;
  int grid;
  // 1: FP64 operands multiplied and summed in double-float (~48-bit significands) on
  // the FP32 pipes; the result is stored in FP64
  int df64;
  // Grouped launches (one launch over the same GEMM of several states, blockIdx.y
  // = member): the member's dims array, and the grid that decides the K split and
  // the workspace layout (so that a member gets the split, and the bits, it gets
  // when launched alone on the full grid); 0: gridDim.x
  const int* dims;
  int split_grid;
};

// Hermitian eigen solve + truncation select (one CTA per problem).
struct EigDesc {
  const void* G;     // n x n Hermitian, row-major, ld = n (overwritten)
  void* V;           // n x n workspace (eigenvectors)
  double* lam;       // n sorted eigenvalues (descending), clamped at 0
  DimExpr n;         // problem size
  int n_max;
  // output of the kept eigenvectors
  void* out;         // destination
  int out_mode;      // 0: out[i*k + j] = V[i][j]   (columns as a row-major n x k matrix)
                     // 1: out[j*n + i] = conj(V[i][j])  (k x n, conjugate transpose)
                     // 2: nothing
  int dim_out;       // index into dims where k is written
  double tol;        // relative discarded weight
  DimExpr cap;       // cap on k
  double gap;        // degeneracy gap
  int max_sweeps;
  double* kept_weight;  // optional: sum of kept eigenvalues
  double* total_weight; // optional: sum of all eigenvalues
  double* disc_stat;    // optional: running max of discarded relative weight
  int* err;             // error flags (bit 0: no convergence, bit 1: non-finite)
  double* solver_stats; // optional counters (see qlb_ctx::d_solver)
  int* gate;            // optional: when set, the eigen-solve runs only if *gate != 0
                        // (the zip-up range basis sets it when its cap was reached)
  // grouped launches (blockIdx.y = member): the member's dims array and workspace
  int* dims;
  void* work;
};

// ------------------------------------------------------------------ error plumbing

void set_error(const std::string& msg);
const char* get_error();

#define QLB_CUDA_TRY(expr)                                                                   \
  do {                                                                                       \
    cudaError_t _e = (expr);                                                                 \
    if (_e != cudaSuccess) {                                                                 \
      ::qlb::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));                  \
      return _e == cudaErrorMemoryAllocation ? QLB_ENOMEM : QLB_EDEVICE;                    \
    }                                                                                        \
  } while (0)

}  // namespace qlb
