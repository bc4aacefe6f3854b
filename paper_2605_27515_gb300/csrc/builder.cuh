// Builder and memory helpers shared by the C-ABI and the step.
#pragma once

#include <map>
#include <utility>
#include <vector>

#include "qlb_objects.cuh"

namespace qlb {

qlb_status dev_alloc(qlb_ctx* ctx, void** p, size_t bytes);
void dev_free(qlb_ctx* ctx, void* p);
std::map<void*, std::pair<size_t, qlb_ctx*>>& g_alloc_sizes();

template <typename R>
cudaError_t launch_gemm(const GemmDesc& g, const int* d_dims, cudaStream_t s, double* prof);
// workspace of the work-distributed GEMM for a grid of `grid` CTAs (complex elements;
// its counters must start at zero), and the default grid (two CTAs per SM)
size_t gemm_workspace_elems(int grid);
int gemm_grid_default();
template <typename R>
cudaError_t launch_eig(const EigDesc& e, const int* d_dims, cudaStream_t s, void* work, double* prof);
template <typename R>
cudaError_t launch_eig_kind(int kind, const EigDesc& e, const int* d_dims, cudaStream_t s, void* work, double* prof);
template <typename R>
size_t eig_smem_bytes(int n_max);
// device workspace (complex elements) the eigen-solvers need beyond shared memory
size_t eig_workspace_elems(int n_max);
void init_kernel_attributes();
// zip-up range basis by column-pivoted Gram-Schmidt on the Gram matrix (U and the
// kept count as launch_eig writes them; the gate tells the Jacobi behind it to run)
template <typename R>
cudaError_t launch_zipqr(const EigDesc& e, const int* d_dims, cudaStream_t s, void* work, double* prof);
size_t zipqr_workspace_elems(int n_max);
void init_qr_attributes();
// a named truncation solver in FP64 or double-float (solver numbering of qlb_eig_check)
cudaError_t launch_solver(bool mixed, int solver, const EigDesc& e, const int* d_dims, cudaStream_t s, void* work);
// split-K factor of a (m x m, K) Gram GEMM: the tuned table if it has the bucket,
// else the built-in rule (about 64 CTAs)
int gram_splitk(const qlb_ctx* ctx, long m, long K);
// 3xTF32 complex GEMM on the tensor cores (same descriptor as launch_gemm); err bit 2
// is set when a bounded wait of the kernel gave up
cudaError_t launch_gemm_tc(const GemmDesc& g, const int* d_dims, cudaStream_t s, int* err, double* prof);
size_t tc_gemm_smem_bytes();
// grouped launches: the same launch of S states at once (blockIdx.y = member), the
// member descriptors in device memory (d_grp[S]); n_max = the largest planned size
cudaError_t launch_gemm_group(const GemmDesc* d_grp, int S, int use_df, cudaStream_t s, double* prof);
template <typename R>
cudaError_t launch_eig_group(int n_max, const EigDesc* d_grp, int S, cudaStream_t s, double* prof);
size_t eig_group_workspace_elems(int n_max, int group_n_max);
template <typename R>
cudaError_t launch_zipqr_group(int n_max, const EigDesc* d_grp, int S, cudaStream_t s, double* prof);
void init_tc_attributes();

qlb_status svd_osj(qlb_ctx* ctx, zd* X, int m, int n, double tol, int cap, zd** U, int u_scale, zd** Rr,
                   int r_unscale, int* k_out, int max_sweeps);
qlb_status tt_svd(qlb_ctx* ctx, zd* T, int L, int P, double tol, int cap, std::vector<zd*>& cores,
                  std::vector<int>& D);
void mpo_clear(qlb_ctx* ctx, Mpo& W);
qlb_status make_identity_mpo(qlb_ctx* ctx, int R, Mpo& W);
qlb_status mpo_from_dense(qlb_ctx* ctx, const zd* F, int R, double tol, int cap, Mpo& W);
void mpo_concat(Mpo& A, Mpo& B);
qlb_status mpo_scale(qlb_ctx* ctx, Mpo& W, zd c);
qlb_status mpo_copy(qlb_ctx* ctx, const Mpo& A, Mpo& B);
qlb_status mpo_stack(qlb_ctx* ctx, const std::vector<const Mpo*>& parts, const std::vector<int>& row_off, int D0,
                     Mpo& out);
qlb_status mpo_compress(qlb_ctx* ctx, Mpo& W, double tol, int cap);
qlb_status make_factor(qlb_ctx* ctx, int N, const qlb_factor& f, zd** out);
qlb_status dense_mul(qlb_ctx* ctx, const zd* A, int opA, const zd* B, int N, zd** out);
double dense_inf_norm(qlb_ctx* ctx, const zd* A, int N);
qlb_status mpo_from_terms(qlb_system* sys, const std::vector<DevTerm>& terms, double tol, int cap, Mpo& out);

}  // namespace qlb
