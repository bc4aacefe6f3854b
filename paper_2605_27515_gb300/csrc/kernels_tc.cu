// Complex GEMM on the 5th-generation tensor cores (tcgen05.mma kind::tf32) in
// 3xTF32 split precision with FP32 accumulation in tensor memory: the MPO
// application of the mixed form (the two contractions of every zip-up site,
// Sec. V.A / V.B) runs here, while Gram matrices, eigen-solves, the cutoff and the
// renormalisation stay in FP64 (or double-float) elsewhere.
//
// The descriptor is the one of the FP64 batched GEMM (GemmDesc: op(A) m x k, op(B)
// k x n, batch strides, device-side DimExpr shapes), so the two engines are
// interchangeable launch by launch.
//
// Complex product as one real product.  With A stored as interleaved (re, im)
// pairs, row i of op(A) is already the real row [Ar_i0, Ai_i0, Ar_i1, Ai_i1, ...]
// of length 2k.  The B operand is expanded per complex entry b = B(k, j) into the
// 2 x 2 real block (rows 2j, 2j+1 of the K-major operand, columns 2k, 2k+1)
//      [ Br  -Bi ]
//      [ Bi   Br ]
// so that D[i][2j] = sum Ar Br - Ai Bi = Re C and D[i][2j+1] = sum Ar Bi + Ai Br = Im C:
// the accumulator columns come out in the interleaved complex layout of C.
//
// 3xTF32: every operand value x is split into hi = tf32(x) and lo = tf32(x - hi);
// the product is hi*hi + hi*lo + lo*hi (the lo*lo term is below the FP32
// accumulator's rounding), about 21 bits of each operand.
//
// Tile: 128 rows of C x 64 complex columns (MMA M = 128, N = 128 real columns),
// 16 complex k per stage (32 real K = four K = 8 MMAs per split product), two
// stages.  256 threads: all of them convert FP64 operands into the shared-memory
// tiles (the canonical K-major layout without swizzling: 8-row x 16-byte core
// matrices, K-adjacent core matrices 128 bytes apart, 8-row groups 1024 bytes
// apart), each thread writing whole 16-byte core-matrix rows so that a warp stores
// 512 contiguous bytes (no bank conflicts); thread 0 issues the MMAs and commits
// them to the stage's mbarrier; for the epilogue the two warps of each TMEM lane
// quarter read back half of the accumulator columns each with tcgen05.ld.
// Every mbarrier wait is bounded: on expiry the kernel records an error flag,
// frees its tensor memory and leaves the tile unwritten.

#include <stdint.h>

#include "qlb_internal.cuh"

namespace qlb {

namespace {

constexpr int TC_BM = 128;        // rows of C per CTA (MMA M)
constexpr int TC_BNC = 64;        // complex columns of C per CTA (MMA N = 128)
constexpr int TC_BKC = 16;        // complex k per stage (32 real K)
constexpr int TC_THREADS = 256;
constexpr int TC_TILE_BYTES = 128 * 32 * 4;  // one 128 x 32 TF32 operand tile
constexpr int TC_STAGE_BYTES = 4 * TC_TILE_BYTES;  // A hi, A lo, B hi, B lo
constexpr int TC_SMEM_BYTES = 2 * TC_STAGE_BYTES + 1024 + 64;
constexpr long TC_WAIT_LIMIT = 1L << 24;  // polls of an mbarrier before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// hi = tf32(f), lo = tf32(f - hi) with f the FP32 rounding of x (FP32 bit patterns).
// The split runs in FP32 after one conversion: this GPU's FP64 pipe is narrow, and
// f already carries the ~22 bits that hi + lo keep.
__device__ __forceinline__ void split3(double x, uint32_t& hi, uint32_t& lo) {
  const float f = __double2float_rn(x);
  hi = to_tf32(f);
  lo = to_tf32(f - __uint_as_float(hi));
}

// byte offset of element (row r, real k c) in a 128 x 32 K-major tile
__device__ __forceinline__ uint32_t tile_off(int r, int c) {
  return (uint32_t)(((r >> 3) << 10) + ((c >> 2) << 7) + ((r & 7) << 4) + ((c & 3) << 2));
}

// shared-memory matrix descriptor: start, leading-dimension (K) byte offset,
// stride-dimension (M/N) byte offset, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  return d;
}

// instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major, M x N
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok;
}

// bounded wait of thread 0 on an mbarrier phase; returns 0 when it gave up
__device__ __forceinline__ int mbar_wait_bounded(uint32_t addr, uint32_t parity) {
  for (long it = 0; it < TC_WAIT_LIMIT; it++)
    if (mbar_try_wait(addr, parity)) return 1;
  return 0;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// element (k, j) of op(B)
__device__ __forceinline__ zd load_opb(const zd* B, int op, long ld, int k, int j) {
  if (op == OP_N) return B[(long)k * ld + j];
  zd v = B[(long)j * ld + k];
  if (op == OP_C) v.im = -v.im;
  return v;
}

__device__ __forceinline__ zd load_op(const zd* P, int op, long ld, int i, int k) {
  if (op == OP_N) return P[(long)i * ld + k];
  zd v = P[(long)k * ld + i];
  if (op == OP_C) v.im = -v.im;
  return v;
}

__global__ void __launch_bounds__(TC_THREADS) k_tc_zgemm(GemmDesc g, const int* __restrict__ d, int* err,
                                                         double* prof) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  const int m = dev_eval(g.m, d), n = dev_eval(g.n, d), K = dev_eval(g.k, d);
  const int nb1 = dev_eval(g.nb1, d), nb2 = dev_eval(g.nb2, d);
  const int bz = blockIdx.z;
  if (bz >= nb1 * nb2 || m <= 0 || n <= 0) return;
  const int row0 = blockIdx.y * TC_BM, col0 = blockIdx.x * TC_BNC;
  if (row0 >= m || col0 >= n) return;
  const int b1 = bz / nb2, b2 = bz - b1 * nb2;
  const long lda = dev_eval(g.lda, d), ldb = dev_eval(g.ldb, d), ldc = dev_eval(g.ldc, d);
  const zd* A = (const zd*)g.A + (long)b1 * dev_eval(g.sA1, d) + (long)b2 * dev_eval(g.sA2, d);
  const zd* B = (const zd*)g.B + (long)b1 * dev_eval(g.sB1, d) + (long)b2 * dev_eval(g.sB2, d);
  zd* C = (zd*)g.C + (long)b1 * dev_eval(g.sC1, d) + (long)b2 * dev_eval(g.sC2, d);
  if (prof && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) {
    double nb = (double)(nb1 * nb2);
    atomicAdd(prof, 8.0 * (double)m * (double)n * (double)K * nb);
    atomicAdd(prof + QLB_K_COUNT, 16.0 * ((double)m * K + (double)K * n + (double)m * n) * nb);
  }

  // 1024-byte aligned stage buffers, then two mbarriers and the TMEM address slot
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* mbar = (uint64_t*)(base + 2 * TC_STAGE_BYTES);
  uint32_t* tmem_slot = (uint32_t*)(mbar + 2);
  int* s_fail = (int*)(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_tf32(128, 128);
  const int nchunks = (K + TC_BKC - 1) / TC_BKC;

  for (int ch = 0; ch < nchunks; ch++) {
    const int st = ch & 1;
    unsigned char* sA_hi = base + st * TC_STAGE_BYTES;
    unsigned char* sA_lo = sA_hi + TC_TILE_BYTES;
    unsigned char* sB_hi = sA_lo + TC_TILE_BYTES;
    unsigned char* sB_lo = sB_hi + TC_TILE_BYTES;
    // the MMAs of chunk ch - 2 read this stage: wait for their commit
    if (ch >= 2) {
      if (tid == 0 && !mbar_wait_bounded(smem_u32(&mbar[st]), (uint32_t)(((ch - 2) >> 1) & 1))) *s_fail = 1;
      __syncthreads();
      if (*s_fail) break;
    }
    const int k0 = ch * TC_BKC;
    // A: 128 rows x 16 complex k.  Item (r, cp): complex k = 2cp, 2cp + 1 of row r,
    // i.e. real columns 4cp .. 4cp + 3 = one 16-byte core-matrix row in hi and in lo
    for (int x = tid; x < TC_BM * 8; x += TC_THREADS) {
      const int r = ((x >> 6) << 3) + (x & 7), cp = (x >> 3) & 7;
      const int gi = row0 + r, gk = k0 + 2 * cp;
      zd a0 = mk<double>(0.0, 0.0), a1 = mk<double>(0.0, 0.0);
      if (gi < m) {
        if (gk < K) a0 = load_op(A, g.opA, lda, gi, gk);
        if (gk + 1 < K) a1 = load_op(A, g.opA, lda, gi, gk + 1);
      }
      uint4 h, l;
      split3(a0.re, h.x, l.x);
      split3(a0.im, h.y, l.y);
      split3(a1.re, h.z, l.z);
      split3(a1.im, h.w, l.w);
      const uint32_t o = tile_off(r, 4 * cp);
      *(uint4*)(sA_hi + o) = h;
      *(uint4*)(sA_lo + o) = l;
    }
    // B: 64 complex columns x 16 complex k.  Item (j, cp): b0 = B(2cp, j), b1 = B(2cp+1, j)
    // give real row 2j = [b0.re, -b0.im, b1.re, -b1.im] and row 2j+1 = [b0.im, b0.re,
    // b1.im, b1.re] over real columns 4cp .. 4cp + 3
    for (int x = tid; x < TC_BNC * 8; x += TC_THREADS) {
      const int j = ((x >> 5) << 2) + (x & 3), cp = (x >> 2) & 7;
      const int gj = col0 + j, gk = k0 + 2 * cp;
      zd b0 = mk<double>(0.0, 0.0), b1 = mk<double>(0.0, 0.0);
      if (gj < n) {
        if (gk < K) b0 = load_opb(B, g.opB, ldb, gk, gj);
        if (gk + 1 < K) b1 = load_opb(B, g.opB, ldb, gk + 1, gj);
      }
      uint32_t r0h, r0l, i0h, i0l, n0h, n0l, r1h, r1l, i1h, i1l, n1h, n1l;
      split3(b0.re, r0h, r0l);
      split3(b0.im, i0h, i0l);
      split3(-b0.im, n0h, n0l);
      split3(b1.re, r1h, r1l);
      split3(b1.im, i1h, i1l);
      split3(-b1.im, n1h, n1l);
      const uint32_t o0 = tile_off(2 * j, 4 * cp), o1 = tile_off(2 * j + 1, 4 * cp);
      *(uint4*)(sB_hi + o0) = make_uint4(r0h, n0h, r1h, n1h);
      *(uint4*)(sB_lo + o0) = make_uint4(r0l, n0l, r1l, n1l);
      *(uint4*)(sB_hi + o1) = make_uint4(i0h, r0h, i1h, r1h);
      *(uint4*)(sB_lo + o1) = make_uint4(i0l, r0l, i1l, r1l);
    }
    // make the generic-proxy stores visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t aH = smem_u32(sA_hi), aL = smem_u32(sA_lo), bH = smem_u32(sB_hi), bL = smem_u32(sB_lo);
#pragma unroll
      for (int kk = 0; kk < 4; kk++) {
        const uint32_t o = kk * 256;  // two 128-byte core matrices per K = 8
        mma_tf32(tmem, smem_desc(aH + o), smem_desc(bH + o), idesc, (ch > 0 || kk > 0) ? 1u : 0u);
        mma_tf32(tmem, smem_desc(aH + o), smem_desc(bL + o), idesc, 1u);
        mma_tf32(tmem, smem_desc(aL + o), smem_desc(bH + o), idesc, 1u);
      }
      mma_commit(smem_u32(&mbar[st]));
    }
  }
  // wait for the last commit of each stage, so that no arrival is still pending on
  // this CTA's shared memory when it exits (the last one covers every MMA)
  if (tid == 0 && !*s_fail) {
    for (int last = nchunks - 2; last < nchunks; last++)
      if (last >= 0 && !mbar_wait_bounded(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1))) *s_fail = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool fail = *s_fail != 0;
  if (fail) {
    if (tid == 0 && err) atomicOr(err, 4);
  } else {
    zd alpha = mk<double>(g.alpha_re, g.alpha_im);
    if (g.alpha_scale) {
      double sc = *g.alpha_scale;
      if (g.alpha_scale_rsqrt) sc = (sc > 0.0) ? 1.0 / sqrt(sc) : 0.0;
      alpha = cscale(alpha, sc);
    }
    const int quarter = warp & 3;               // TMEM lanes 32 quarter .. 32 quarter + 31
    const int row = row0 + quarter * 32 + lane;  // accumulator row = TMEM lane
    for (int cb = (warp >> 2) * 2; cb < (warp >> 2) * 2 + 2; cb++) {
      uint32_t r[32];
      if (nchunks > 0) {
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cb * 32), r);
      } else {
#pragma unroll
        for (int q = 0; q < 32; q++) r[q] = 0u;
      }
      if (row < m) {
#pragma unroll
        for (int q = 0; q < 16; q++) {
          const int gj = col0 + cb * 16 + q;
          if (gj < n) {
            zd v = cmul(alpha, mk<double>((double)__uint_as_float(r[2 * q]), (double)__uint_as_float(r[2 * q + 1])));
            zd* dst = C + (long)row * ldc + gj;
            if (g.beta) v = cadd(v, *dst);
            *dst = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

}  // namespace

size_t tc_gemm_smem_bytes() { return TC_SMEM_BYTES; }

cudaError_t launch_gemm_tc(const GemmDesc& g, const int* d_dims, cudaStream_t s, int* err, double* prof) {
  const int nb = g.nb_max > 0 ? g.nb_max : 1;
  dim3 grid((g.n_max + TC_BNC - 1) / TC_BNC, (g.m_max + TC_BM - 1) / TC_BM, nb);
  if (grid.x == 0 || grid.y == 0) return cudaSuccess;
  k_tc_zgemm<<<grid, TC_THREADS, TC_SMEM_BYTES, s>>>(g, d_dims, err, prof);
  return cudaGetLastError();
}

void init_tc_attributes() {
  cudaFuncSetAttribute(k_tc_zgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BYTES);
}

}  // namespace qlb
