// Tensor-core GEMM for sm_103a: tcgen05.mma with TMEM accumulators, operands staged in
// shared memory by TMA (cp.async.bulk.tensor) through an mbarrier pipeline.
//
// Core product (real):  D[b][i][j] = sum_k A[b][i][k] * B[b][j][k]
// with A (M x K) and B (N x K) both K-major (K contiguous), elements TF32 (stored as FP32)
// or BF16, accumulated in FP32 in tensor memory.  One CTA computes a 128 x BN tile:
//   warp 0 lane 0   issues the TMA loads of A and B k-blocks into a STAGES-deep ring,
//   warp 1 lane 0   issues the tcgen05.mma instructions (4 per 128-byte k-block) and
//                   commits them to the ring's "empty" barriers and, at the end, to the
//                   accumulator barrier,
//   all 4 warps     read the accumulator back with tcgen05.ld (warp w owns TMEM lanes
//                   32w..32w+31, i.e. tile rows 32w..32w+31) and write the output.
// Every wait on an mbarrier is bounded (kWaitNs); a wait that gives up sets the caller's
// error flag and the kernel winds down without touching the output.
//
// Complex products ride on the real core (the paper's contractions, Sec. III.A, are
// complex):  with op(A) = X (m x k) and op(B) = Y (k x n) complex,
//   Ar[i][2p] = Re X_ip, Ar[i][2p+1] = Im X_ip                                   (m x 2k)
//   Br[2q][2p] = Re Y_pq, Br[2q][2p+1] = -Im Y_pq,
//   Br[2q+1][2p] = Im Y_pq, Br[2q+1][2p+1] = Re Y_pq                              (2n x 2k)
// gives Ar Br^T = the interleaved (re, im) m x n result, i.e. one real GEMM of the same
// 8mnk flops as a complex one, written straight into complex64 storage.  Split precision
// (TF32x3 / BF16x3): x = hi(x) + lo(x) with hi, lo in the MMA type; the packed operands
// carry three K-segments, A as [hi | hi | lo] and B as [hi | lo | hi], so one GEMM over
// 3 x 2k sums hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding for TF32).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "tcgemm.h"

namespace mpdo {
std::atomic<long long> g_tc_launches{0};
namespace tc {

constexpr int BM = 128;
constexpr int kThreads = 128;
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s per wait, then give up

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = gtime();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_test(bar, parity)) return true;
    if (gtime() - t0 > kWaitNs) return false;
  }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4, %5}], [%2];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor of a K-major tile written by TMA with 128-byte swizzle:
// rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), version 1
// (tcgen05), layout SWIZZLE_128B.  The leading byte offset is not used by this layout.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor, dense kind::tf32 / kind::f16: D format F32 (bits 4-5 = 1), A and
// B formats (bits 7-9, 10-12: TF32 = 2, BF16 = 1), both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24.
template <int ELT>
__host__ __device__ constexpr uint32_t idesc(int n) {
  return (1u << 4) | ((ELT == 4 ? 2u : 1u) << 7) | ((ELT == 4 ? 2u : 1u) << 10) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
template <int ELT>
__device__ __forceinline__ void umma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t id,
                                     uint32_t accum) {
  if constexpr (ELT == 4) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(id), "r"(accum));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(id), "r"(accum));
  }
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(bar))
      : "memory");
}
// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

struct Epi {
  float* d;       // output, real view: row i of batch b at d + b*sd + i*ldd (floats)
  long ldd, sd;
  double* d64;    // FP64 accumulation target (mode 1), same strides
  float ar, ai;   // complex alpha (pairs of columns are (re, im)); mode 0
  float br, bi;   // complex beta; use_beta = 0 skips reading d
  int use_beta;
  double scale;   // mode 1: d64 += scale * acc
  int mode;       // 0: FP32 (complex alpha/beta), 1: FP64 accumulate
};

template <int ELT, int BN, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap mb,
                   int M, int N, int K, Epi ep, int* err) {
  constexpr int BK = 128 / ELT;                      // elements per 128-byte k-block row
  constexpr uint32_t A_BYTES = BM * 128, B_BYTES = BN * 128;
  constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
  extern __shared__ uint8_t smem_raw[];
  // tiles on a 1024-byte boundary (the 128-byte swizzle pattern repeats every 8 rows)
  uint8_t* smem = smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accb = empty + STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accb + 1);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM, bz = blockIdx.z;
  const int nk = (K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accb, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      // producer: k-block kb goes to stage kb % STAGES once the MMAs of kb - STAGES are done
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1)) {
          atomicExch(abort_flag, 1);
          atomicExch(err, 1);
          break;
        }
        if (*(volatile int*)abort_flag) break;
        uint8_t* sa = smem + s * STAGE_BYTES;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        tma_load_3d(sa, &ma, &full[s], kb * BK, m0, bz);
        tma_load_3d(sa + A_BYTES, &mb, &full[s], kb * BK, n0, bz);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t id = idesc<ELT>(BN);
      bool ok = true;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        if (!mbar_wait(&full[s], (kb / STAGES) & 1)) {
          atomicExch(abort_flag, 1);
          atomicExch(err, 2);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = su32(smem + s * STAGE_BYTES);
        const uint64_t ad = sdesc(sa), bd = sdesc(sa + A_BYTES);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)   // 32 bytes of K per instruction
          umma<ELT>(tmem, ad + 2 * kk, bd + 2 * kk, id, (kb | kk) != 0);
        umma_commit(&empty[s]);
      }
      // the accumulator barrier fires when every MMA issued above has completed
      umma_commit(accb);
      (void)ok;
    }
    __syncwarp();
  }

  // epilogue: TMEM -> registers -> global
  bool ready = true;
  if (lane == 0) ready = mbar_wait(accb, 0);
  ready = __shfl_sync(0xffffffffu, ready ? 1 : 0, 0) != 0;
  if (!ready) {
    if (lane == 0) atomicExch(err, 3);
  } else if (!*(volatile int*)abort_flag) {
    tc_fence_after();
    const int row = m0 + warp * 32 + lane;
    const uint32_t tw = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c = 0; c < BN; c += 32) {
      float v[32];
      tmem_ld32(tw + c, v);
      if (row < M) {
        const int col0 = n0 + c;
        if (ep.mode == 0) {
          float* dp = ep.d + (long)bz * ep.sd + (long)row * ep.ldd + col0;
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            if (col0 + j >= N) break;
            const float xr = v[j], xi = v[j + 1];
            float yr = ep.ar * xr - ep.ai * xi, yi = ep.ar * xi + ep.ai * xr;
            if (ep.use_beta) {
              const float cr = dp[j], ci = (col0 + j + 1 < N) ? dp[j + 1] : 0.f;
              yr += ep.br * cr - ep.bi * ci;
              yi += ep.br * ci + ep.bi * cr;
            }
            dp[j] = yr;
            if (col0 + j + 1 < N) dp[j + 1] = yi;
          }
        } else {
          double* dp = ep.d64 + (long)bz * ep.sd + (long)row * ep.ldd + col0;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (col0 + j < N) dp[j] += ep.scale * (double)v[j];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------------ operand packing
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
template <typename TO>
__device__ __forceinline__ void split3(float x, TO& hi, TO& lo);
template <>
__device__ __forceinline__ void split3<float>(float x, float& hi, float& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - hi);
}
template <>
__device__ __forceinline__ void split3<__nv_bfloat16>(float x, __nv_bfloat16& hi,
                                                      __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}
template <typename TO>
__device__ __forceinline__ TO to_elt(float x);
template <>
__device__ __forceinline__ float to_elt<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_elt<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}

// X[r][c] = src[b*sb + r*s_r + c*s_c] (conjugated when conj), r < rows, c < kc.
// side 0 (A operand): out[b][r][t*2kc + 2c + {0,1}] = parts of (Re, Im)
// side 1 (B operand): out[b][2r][t*2kc + 2c + {0,1}] = parts of (Re, -Im),
//                     out[b][2r+1][...]             = parts of (Im, Re)
// parts t: nparts = 1 -> the value; nparts = 3 -> A [hi, hi, lo], B [hi, lo, hi].
constexpr int PT = 32;
template <typename TIN, typename TO>
__global__ void __launch_bounds__(PT * 8)
    pack_kernel(int rows, int kc, const TIN* __restrict__ src, long s_r, long s_c, long sb,
                int conj, int side, int nparts, TO* __restrict__ out, long ldo, long so) {
  __shared__ float2 tile[PT][PT + 1];   // [r][c]
  const int r0 = blockIdx.y * PT, c0 = blockIdx.x * PT, b = blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;
  src += (long)b * sb;
  const bool c_fast = (s_c == 1);
  for (int q = ty; q < PT; q += 8) {
    // coalesced along whichever index is contiguous in the source
    const int r = c_fast ? r0 + q : r0 + tx;
    const int c = c_fast ? c0 + tx : c0 + q;
    float2 v = make_float2(0.f, 0.f);
    if (r < rows && c < kc) {
      const TIN t = src[(long)r * s_r + (long)c * s_c];
      v = make_float2((float)t.x, conj ? -(float)t.y : (float)t.y);
    }
    if (c_fast) tile[q][tx] = v; else tile[tx][q] = v;
  }
  __syncthreads();
  const long kseg = 2L * kc;
  for (int q = ty; q < PT; q += 8) {
    const int r = r0 + q, c = c0 + tx;
    if (r >= rows || c >= kc) continue;
    const float2 v = tile[q][tx];
    if (side == 0) {
      TO* o = out + (long)b * so + (long)r * ldo + 2L * c;
      if (nparts == 1) {
        o[0] = to_elt<TO>(v.x);
        o[1] = to_elt<TO>(v.y);
      } else {
        TO hr, lr, hi, li;
        split3<TO>(v.x, hr, lr);
        split3<TO>(v.y, hi, li);
        o[0] = hr; o[1] = hi;
        o[kseg] = hr; o[kseg + 1] = hi;
        o[2 * kseg] = lr; o[2 * kseg + 1] = li;
      }
    } else {
      TO* o0 = out + (long)b * so + (2L * r) * ldo + 2L * c;
      TO* o1 = o0 + ldo;
      if (nparts == 1) {
        o0[0] = to_elt<TO>(v.x); o0[1] = to_elt<TO>(-v.y);
        o1[0] = to_elt<TO>(v.y); o1[1] = to_elt<TO>(v.x);
      } else {
        TO hr, lr, hi, li, hm, lm;
        split3<TO>(v.x, hr, lr);
        split3<TO>(v.y, hi, li);
        split3<TO>(-v.y, hm, lm);
        o0[0] = hr; o0[1] = hm; o1[0] = hi; o1[1] = hr;
        o0[kseg] = lr; o0[kseg + 1] = lm; o1[kseg] = li; o1[kseg + 1] = lr;
        o0[2 * kseg] = hr; o0[2 * kseg + 1] = hm; o1[2 * kseg] = hi; o1[2 * kseg + 1] = hr;
      }
    }
  }
}

// ------------------------------------------------------------------ exact products
// FP64-accurate product of FP32 operands on the BF16 tensor cores, by error-free slicing
// (the splitting scheme of Ozaki, Ogita, Oishi and Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012).  Every row r of the A operand (and of the
// B operand) is scaled by 2^-e_r, e_r the exponent of its largest |Re|, |Im|, and written as
// six slices of integers in [-128, 128] (exact in BF16):
//   x 2^-e_r = 2^-7 (q_1 + 2^-8 q_2 + ... + 2^-40 q_6) + O(2^-48).
// The product of slice t of A and slice u of B is a sum of integer products of at most
// 2^14 each; over a chunk of 1024 real K terms it stays below 2^24 and is therefore exact in
// the FP32 accumulator.  Each chunk's accumulator is drained into FP64 registers with the
// weight 2^-(14 + 8(t+u)) (t, u from 0) and, at the end, scaled by 2^(e_r + e_q).  The slice
// pairs with t + u <= 5 are computed (21 of 36): a dropped pair contributes terms below
// 2^-48 of the two rows' largest entries.  The result carries the FP32 inputs' product to
// ~2^-48 of the rows' largest entries, enough for the eigenvalues of a Gram matrix of FP32
// data down to ~1e-14 of the largest (the floor of FP64 sums of the same products).
constexpr int XS = 6;          // slices per operand
constexpr int XPAIRS = 21;     // slice pairs (t, u) with t + u <= XS - 1
constexpr int XBN = 64;        // output tile width (real columns)
constexpr int XSTAGES = 8;
constexpr int XCHUNK = 16;     // k-blocks of 64 BF16 per exact chunk (1024 real terms)
constexpr int XTHREADS = 192;  // warp 0 TMA, warp 1 MMA, warps 2-5 drain

// pair index -> (t, u), enumerating t = 0.., u = 0..XS-1-t
__device__ __forceinline__ void pair_tu(int p, int& t, int& u) {
  t = 0;
  while (p >= XS - t) {
    p -= XS - t;
    ++t;
  }
  u = p;
}

__global__ void __launch_bounds__(XTHREADS, 1)
    tc_exact_kernel(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap mb,
                    int M, int N, int kr, int ldk, const int* __restrict__ ea,
                    const int* __restrict__ eb, double* C, long ldc, long sc, int accumulate,
                    int* err) {
  constexpr uint32_t A_BYTES = BM * 128, B_BYTES = XBN * 128;
  constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + XSTAGES * STAGE_BYTES);
  uint64_t* empty = full + XSTAGES;
  uint64_t* tfull = empty + XSTAGES;   // [2] accumulator buffer ready for the drain
  uint64_t* tempty = tfull + 2;        // [2] accumulator buffer drained
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + 2);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * XBN, m0 = blockIdx.y * BM, bz = blockIdx.z;
  const int nkb = (kr + 63) / 64;                  // k-blocks per slice pair
  const int nch = (nkb + XCHUNK - 1) / XCHUNK;     // exact chunks per slice pair
  const int total_chunks = XPAIRS * nch;

  if (threadIdx.x == 0) {
    for (int s = 0; s < XSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tslot)),
                 "r"(2 * XBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int ch = 0; ch < total_chunks && !*(volatile int*)abort_flag; ++ch) {
        const int pair = ch / nch, c = ch % nch;
        int t, u;
        pair_tu(pair, t, u);
        const int kb1 = min(nkb, (c + 1) * XCHUNK);
        for (int kb = c * XCHUNK; kb < kb1; ++kb, ++it) {
          const int s = it % XSTAGES;
          if (it >= XSTAGES && !mbar_wait(&empty[s], ((it / XSTAGES) - 1) & 1)) {
            atomicExch(abort_flag, 1);
            atomicExch(err, 11);
            break;
          }
          uint8_t* sa = smem + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          tma_load_3d(sa, &ma, &full[s], t * ldk + kb * 64, m0, bz);
          tma_load_3d(sa + A_BYTES, &mb, &full[s], u * ldk + kb * 64, n0, bz);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t id = idesc<2>(XBN);
      int it = 0;
      for (int ch = 0; ch < total_chunks; ++ch) {
        const int c = ch % nch, buf = ch & 1;
        // the drain of chunk ch - 2 must have emptied this accumulator buffer
        if (ch >= 2 && !mbar_wait(&tempty[buf], ((ch >> 1) - 1) & 1)) {
          atomicExch(abort_flag, 1);
          atomicExch(err, 12);
          break;
        }
        tc_fence_after();
        const uint32_t td = tmem + buf * XBN;
        const int kb1 = min(nkb, (c + 1) * XCHUNK);
        bool ok = true;
        for (int kb = c * XCHUNK; kb < kb1; ++kb, ++it) {
          const int s = it % XSTAGES;
          if (!mbar_wait(&full[s], (it / XSTAGES) & 1)) {
            atomicExch(abort_flag, 1);
            atomicExch(err, 13);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = su32(smem + s * STAGE_BYTES);
          const uint64_t ad = sdesc(sa), bd = sdesc(sa + A_BYTES);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            umma<2>(td, ad + 2 * kk, bd + 2 * kk, id, (kb > c * XCHUNK || kk) ? 1u : 0u);
          umma_commit(&empty[s]);
        }
        if (!ok) break;
        umma_commit(&tfull[buf]);
      }
    }
    __syncwarp();
  } else {
    // drain warps: TMEM lanes 32 (warp % 4) .. +31 are tile rows
    const int q = warp & 3;
    const int row = m0 + q * 32 + lane;
    double acc[XBN];
#pragma unroll
    for (int j = 0; j < XBN; ++j) acc[j] = 0.0;
    bool ok = true;
    for (int ch = 0; ch < total_chunks; ++ch) {
      const int pair = ch / nch, buf = ch & 1;
      int t, u;
      pair_tu(pair, t, u);
      bool ready = true;
      if (lane == 0) ready = mbar_wait(&tfull[buf], (ch >> 1) & 1);
      ready = __shfl_sync(0xffffffffu, ready ? 1 : 0, 0) != 0;
      if (!ready || *(volatile int*)abort_flag) {
        if (lane == 0 && !ready) atomicExch(err, 14);
        ok = false;
        break;
      }
      tc_fence_after();
      const double w = ldexp(1.0, -(14 + 8 * (t + u)));
      const uint32_t tw = tmem + ((uint32_t)(q * 32) << 16) + buf * XBN;
#pragma unroll
      for (int cb = 0; cb < XBN; cb += 32) {
        float v[32];
        tmem_ld32(tw + cb, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[cb + j] = fma(w, (double)v[j], acc[cb + j]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&tempty[buf])) : "memory");
    }
    if (ok && row < M) {
      const int er = ea[(long)bz * M + row];
      double* cp = C + (long)bz * sc + (long)row * ldc;
#pragma unroll
      for (int j = 0; j < XBN; ++j) {
        const int col = n0 + j;
        if (col < N) {
          const double v = ldexp(acc[j], er + eb[(long)bz * (N / 2) + col / 2]);
          cp[col] = accumulate ? cp[col] + v : v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * XBN)
                 : "memory");
  }
}

// e[b][r] = exponent of the largest |Re|, |Im| of row r of X (X[r][c] = src[b*sb + r*s_r +
// c*s_c], c < kc): max = f 2^e with f in [0.5, 1); 0 for an all-zero row.
template <typename TIN>
__global__ void __launch_bounds__(256) row_exp_kernel(int rows, int kc, const TIN* __restrict__ src,
                                                     long s_r, long s_c, long sb, int* e) {
  __shared__ double red[256];
  const int r = blockIdx.x, b = blockIdx.y;
  const TIN* x = src + (long)b * sb + (long)r * s_r;
  double mx = 0.0;
  for (int c = threadIdx.x; c < kc; c += blockDim.x) {
    const TIN v = x[(long)c * s_c];
    mx = fmax(mx, fmax(fabs((double)v.x), fabs((double)v.y)));
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int ex = 0;
    if (red[0] > 0.0) frexp(red[0], &ex);
    e[(long)b * rows + r] = ex;
  }
}

// XS integer slices of x in (-1, 1): x = 2^-7 sum_t 2^-8t q_(t+1) + r, |q| <= 128,
// |r| <= 2^-(8 XS) (every step is exact in FP32: y - rint(y) is a multiple of y's last bit).
template <typename F>
__device__ __forceinline__ void slice_all(F x, float* q) {
  F y = x * (F)128;
#pragma unroll
  for (int t = 0; t < XS; ++t) {
    const F r = rint(y);
    q[t] = (float)r;
    y = (y - r) * (F)256;
  }
}

// Sliced packing (layout as pack_kernel, with XS K-segments of ldk elements, one per slice;
// the segment tails up to ldk are written as zeros): row scale 2^-e[b][r] (A side) or the
// column scale of the complex column (B side, rows 2r and 2r+1).
template <typename TIN>
__global__ void __launch_bounds__(PT * 8)
    pack_exact_kernel(int rows, int kc, const TIN* __restrict__ src, long s_r, long s_c, long sb,
                      int conj, int side, const int* __restrict__ e, __nv_bfloat16* __restrict__ out,
                      long ldo, long so, int ldk) {
  using F = decltype(TIN().x);
  __shared__ TIN tile[PT][PT + 1];
  const int r0 = blockIdx.y * PT, c0 = blockIdx.x * PT, b = blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;
  src += (long)b * sb;
  const bool c_fast = (s_c == 1);
  for (int qq = ty; qq < PT; qq += 8) {
    const int r = c_fast ? r0 + qq : r0 + tx;
    const int c = c_fast ? c0 + tx : c0 + qq;
    TIN v;
    v.x = 0;
    v.y = 0;
    if (r < rows && c < kc) {
      v = src[(long)r * s_r + (long)c * s_c];
      if (conj) v.y = -v.y;
    }
    if (c_fast) tile[qq][tx] = v; else tile[tx][qq] = v;
  }
  __syncthreads();
  for (int qq = ty; qq < PT; qq += 8) {
    const int r = r0 + qq, c = c0 + tx;
    if (r >= rows || c >= kc) continue;
    const int er = e[(long)b * rows + r];
    const TIN v = tile[qq][tx];
    float qr[XS], qi[XS];
    slice_all<F>(ldexp(v.x, -er), qr);
    slice_all<F>(ldexp(v.y, -er), qi);
    if (side == 0) {
      __nv_bfloat16* o = out + (long)b * so + (long)r * ldo + 2L * c;
#pragma unroll
      for (int t = 0; t < XS; ++t) {
        o[t * ldk] = __float2bfloat16_rn(qr[t]);
        o[t * ldk + 1] = __float2bfloat16_rn(qi[t]);
      }
    } else {
      __nv_bfloat16* o0 = out + (long)b * so + (2L * r) * ldo + 2L * c;
      __nv_bfloat16* o1 = o0 + ldo;
#pragma unroll
      for (int t = 0; t < XS; ++t) {
        o0[t * ldk] = __float2bfloat16_rn(qr[t]);
        o0[t * ldk + 1] = __float2bfloat16_rn(-qi[t]);
        o1[t * ldk] = __float2bfloat16_rn(qi[t]);
        o1[t * ldk + 1] = __float2bfloat16_rn(qr[t]);
      }
    }
  }
}

// Zero the K-segment tails [kr, ldk) of every slice of every packed row (rows_out rows).
__global__ void zero_tails_kernel(long rows_out, int kr, int ldk, __nv_bfloat16* out, long ldo) {
  const int w = ldk - kr;
  const long total = rows_out * XS * w;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long r = e / (XS * w);
    const int t = (int)((e / w) % XS), j = (int)(e % w);
    out[r * ldo + (long)t * ldk + kr + j] = __float2bfloat16_rn(0.f);
  }
}

// Real operand packing for the BF16 core: out[r][c] = bf16(src[r*s_r + c*s_c]), r < rows,
// c < kc (row stride ldo elements); tiled through shared memory so that both the read and
// the write are coalesced whichever index is contiguous in the source.
__global__ void __launch_bounds__(PT * 8)
    pack_real_bf16_kernel(int rows, int kc, const float* __restrict__ src, long s_r, long s_c,
                          __nv_bfloat16* __restrict__ out, long ldo) {
  __shared__ float tile[PT][PT + 1];
  const int r0 = blockIdx.y * PT, c0 = blockIdx.x * PT;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool c_fast = (s_c == 1);
  for (int q = ty; q < PT; q += 8) {
    const int r = c_fast ? r0 + q : r0 + tx;
    const int c = c_fast ? c0 + tx : c0 + q;
    const float v = (r < rows && c < kc) ? src[(long)r * s_r + (long)c * s_c] : 0.f;
    if (c_fast) tile[q][tx] = v; else tile[tx][q] = v;
  }
  __syncthreads();
  for (int q = ty; q < PT; q += 8) {
    const int r = r0 + q, c = c0 + tx;
    if (r < rows && c < kc) out[(long)r * ldo + c] = __float2bfloat16_rn(tile[q][tx]);
  }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// 3-D K-major map: dims {K, rows, batch}, box {128 bytes of K, box_rows, 1}.
bool make_map(CUtensorMap* map, int elt, const void* base, long k, long rows, long ld, long sb,
              int batch, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows, (cuuint64_t)batch};
  const cuuint64_t strides[2] = {(cuuint64_t)ld * elt,
                                 (cuuint64_t)(batch > 1 ? sb : rows * ld) * elt};
  const cuuint32_t box[3] = {(cuuint32_t)(128 / elt), (cuuint32_t)box_rows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(map, elt == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                  3, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int ELT, int BN, int STAGES>
constexpr size_t smem_bytes() {
  return (size_t)STAGES * (BM + BN) * 128 + 1024 + 2 * STAGES * 8 + 64;
}

template <int ELT, int BN, int STAGES>
cudaError_t launch_bn(cudaStream_t st, const CUtensorMap& ma, const CUtensorMap& mb, int M, int N,
                      int K, int batch, const Epi& ep, int* err) {
  constexpr size_t sm = smem_bytes<ELT, BN, STAGES>();
  static const cudaError_t attr = cudaFuncSetAttribute(
      tc_gemm_kernel<ELT, BN, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (attr != cudaSuccess) return attr;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  tc_gemm_kernel<ELT, BN, STAGES><<<grid, kThreads, sm, st>>>(ma, mb, M, N, K, ep, err);
  count_launch();
  g_tc_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace tc

using namespace tc;

int tc_pick_bn(long M, long N, int batch) {
  const long mt = (M + BM - 1) / BM;
  const long t256 = mt * ((N + 255) / 256) * batch, t128 = mt * ((N + 127) / 128) * batch;
  if (N > 128 && t256 >= 148) return 256;
  if (N > 64 && t128 >= 74) return 128;
  return 64;
}

cudaError_t tc_gemm_real(cudaStream_t st, int elt, int M, int N, int K, const void* A, long lda,
                         long sa, const void* B, long ldb, long sb, int batch, const TcEpilogue& e,
                         int* err, int bn) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (K <= 0) return cudaErrorInvalidValue;
  if ((lda * elt) % 16 || (ldb * elt) % 16 || (batch > 1 && ((sa * elt) % 16 || (sb * elt) % 16)) ||
      (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
    return cudaErrorInvalidValue;
  if (bn <= 0) bn = tc_pick_bn(M, N, batch);
  CUtensorMap ma, mb;
  if (!make_map(&ma, elt, A, K, M, lda, sa, batch, BM) ||
      !make_map(&mb, elt, B, K, N, ldb, sb, batch, bn))
    return cudaErrorInvalidValue;
  Epi ep;
  ep.d = e.d;
  ep.d64 = e.d64;
  ep.ldd = e.ldd;
  ep.sd = e.sd;
  ep.ar = e.ar; ep.ai = e.ai; ep.br = e.br; ep.bi = e.bi;
  ep.use_beta = e.use_beta;
  ep.scale = e.scale;
  ep.mode = e.d64 ? 1 : 0;
  if (elt == 4) {
    if (bn == 256) return launch_bn<4, 256, 4>(st, ma, mb, M, N, K, batch, ep, err);
    if (bn == 128) return launch_bn<4, 128, 6>(st, ma, mb, M, N, K, batch, ep, err);
    return launch_bn<4, 64, 8>(st, ma, mb, M, N, K, batch, ep, err);
  }
  if (bn == 256) return launch_bn<2, 256, 4>(st, ma, mb, M, N, K, batch, ep, err);
  if (bn == 128) return launch_bn<2, 128, 6>(st, ma, mb, M, N, K, batch, ep, err);
  return launch_bn<2, 64, 8>(st, ma, mb, M, N, K, batch, ep, err);
}

size_t tc_pack_bytes(int mode, long rows, long k, int batch) {
  const int elt = tc_mode_elt(mode);
  const long kr = (long)tc_mode_parts(mode) * 2 * k;
  const long ld = tc_pack_ld(mode, k);
  (void)kr;
  return (size_t)batch * rows * ld * elt + 256;
}

template <typename TIN>
cudaError_t tc_pack(cudaStream_t st, int mode, int side, int rows, int kc, const cx<TIN>* src,
                    long s_r, long s_c, long sb, int conj, int batch, void* out) {
  const long ld = tc_pack_ld(mode, kc);
  const long so = (long)(side == 0 ? rows : 2 * rows) * ld;
  dim3 grid((kc + PT - 1) / PT, (rows + PT - 1) / PT, batch), block(PT, 8);
  const int np = tc_mode_parts(mode);
  if (tc_mode_elt(mode) == 4)
    pack_kernel<cx<TIN>, float><<<grid, block, 0, st>>>(rows, kc, src, s_r, s_c, sb, conj, side,
                                                       np, static_cast<float*>(out), ld, so);
  else
    pack_kernel<cx<TIN>, __nv_bfloat16><<<grid, block, 0, st>>>(
        rows, kc, src, s_r, s_c, sb, conj, side, np, static_cast<__nv_bfloat16*>(out), ld, so);
  count_launch();
  return cudaGetLastError();
}

// Source strides of op(X) as an (rows x kc) matrix indexed [r][c] from a row-major matrix
// with leading dimension ld: for the A operand rows = m, c = k; for B rows = n, c = k.
static void op_strides(int side, int op, long ld, long* s_r, long* s_c, int* conj) {
  // A: op(A)[i][p]; N: A[i][p], T/C: A[p][i], R: conj A[i][p]
  // B: X[q][p] = op(B)[p][q]; N/R: B[p][q] -> s_r = 1, s_c = ld; T/C: B[q][p]
  const bool trans = (op == OP_T || op == OP_C);
  *conj = (op == OP_C || op == OP_R) ? 1 : 0;
  const bool rowmajor_rc = side == 0 ? !trans : trans;
  if (rowmajor_rc) { *s_r = ld; *s_c = 1; } else { *s_r = 1; *s_c = ld; }
}

template <typename TIN>
cudaError_t tc_cgemm(cudaStream_t st, int mode, int opa, int opb, int m, int n, int k,
                     const cx<TIN>* A, long lda, long sa, const cx<TIN>* B, long ldb, long sb,
                     float2* C, long ldc, long sc, int batch, float2 alpha, float2 beta,
                     void* ws, size_t ws_bytes, int* err) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  const int elt = tc_mode_elt(mode);
  // K is processed in chunks whose packed operands fit the workspace; later chunks add to
  // the output (beta = 1)
  long kc = k;
  while (kc > 32 && tc_cgemm_ws_bytes(mode, m, n, kc, batch) > ws_bytes) kc = (kc + 1) / 2;
  if (kc < k) kc = std::max(32L, kc / 32 * 32);
  if (tc_cgemm_ws_bytes(mode, m, n, kc, batch) > ws_bytes) return cudaErrorMemoryAllocation;
  long sra, sca, srb, scb;
  int cja, cjb;
  op_strides(0, opa, lda, &sra, &sca, &cja);
  op_strides(1, opb, ldb, &srb, &scb, &cjb);
  for (long k0 = 0; k0 < k; k0 += kc) {
    const int kn = (int)std::min<long>(kc, k - k0);
    const long ld = tc_pack_ld(mode, kn);
    const size_t abytes = ((size_t)batch * m * ld * elt + 255) & ~(size_t)255;
    char* pa = static_cast<char*>(ws);
    char* pb = pa + abytes;
    MPDO_CUDA_TRY(tc_pack<TIN>(st, mode, 0, m, kn, A + k0 * sca, sra, sca, sa, cja, batch, pa));
    MPDO_CUDA_TRY(tc_pack<TIN>(st, mode, 1, n, kn, B + k0 * scb, srb, scb, sb, cjb, batch, pb));
    TcEpilogue e;
    e.d = reinterpret_cast<float*>(C);
    e.ldd = 2 * ldc;
    e.sd = 2 * sc;
    e.ar = alpha.x; e.ai = alpha.y;
    if (k0 == 0) {
      e.br = beta.x; e.bi = beta.y;
    } else {
      e.br = 1.f; e.bi = 0.f;
    }
    e.use_beta = (e.br != 0.f || e.bi != 0.f);
    const long kr = (long)tc_mode_parts(mode) * 2 * kn;
    MPDO_CUDA_TRY(tc_gemm_real(st, elt, m, 2 * n, (int)kr, pa, ld, (long)m * ld, pb, ld,
                               2L * n * ld, batch, e, err, 0));
  }
  return cudaSuccess;
}

// ---- exact products: C (complex FP64) = op(A) op(B), FP32 complex A and B
static size_t exact_bytes(long m, long n, long kc, int batch) {
  const long ldk = (2 * kc + 63) / 64 * 64;
  const size_t a = ((size_t)batch * m * XS * ldk * 2 + 255) & ~(size_t)255;
  const size_t b = ((size_t)batch * 2 * n * XS * ldk * 2 + 255) & ~(size_t)255;
  return a + b + ((size_t)batch * (m + n) * sizeof(int) + 256);
}

size_t tc_exact_ws_bytes(long m, long n, long k, int batch) {
  return exact_bytes(m, n, std::min<long>(k, 4096), batch);
}

cudaError_t tc_exact_init() {
  static const cudaError_t attr = cudaFuncSetAttribute(
      tc_exact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)(XSTAGES * (BM + XBN) * 128 + 1024 + 256));
  return attr;
}

template <typename TA, typename TB>
cudaError_t tc_cgemm_exact(cudaStream_t st, int opa, int opb, int m, int n, int k, const TA* A,
                           long lda, long sa, const TB* B, long ldb, long sb, double2* C, long ldc,
                           long sc, int batch, void* ws, size_t ws_bytes, int* err) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  if (k <= 0) return cudaErrorInvalidValue;
  long kc = k;
  while (kc > 64 && exact_bytes(m, n, kc, batch) > ws_bytes) kc = (kc + 1) / 2;
  if (kc < k) kc = std::max(64L, kc / 64 * 64);
  if (exact_bytes(m, n, kc, batch) > ws_bytes) return cudaErrorMemoryAllocation;
  long sra, sca, srb, scb;
  int cja, cjb;
  op_strides(0, opa, lda, &sra, &sca, &cja);
  op_strides(1, opb, ldb, &srb, &scb, &cjb);
  MPDO_CUDA_TRY(tc_exact_init());
  for (long k0 = 0; k0 < k; k0 += kc) {
    const int kn = (int)std::min<long>(kc, k - k0);
    const int kr = 2 * kn;
    const int ldk = (kr + 63) / 64 * 64;
    const long ldo = (long)XS * ldk;
    char* p = static_cast<char*>(ws);
    __nv_bfloat16* pa = reinterpret_cast<__nv_bfloat16*>(p);
    p += ((size_t)batch * m * ldo * 2 + 255) & ~(size_t)255;
    __nv_bfloat16* pb = reinterpret_cast<__nv_bfloat16*>(p);
    p += ((size_t)batch * 2 * n * ldo * 2 + 255) & ~(size_t)255;
    int* ea = reinterpret_cast<int*>(p);
    int* eb = ea + (size_t)batch * m;
    const TA* a0 = A + k0 * sca;
    const TB* b0 = B + k0 * scb;
    row_exp_kernel<TA><<<dim3(m, batch), 256, 0, st>>>(m, kn, a0, sra, sca, sa, ea);
    row_exp_kernel<TB><<<dim3(n, batch), 256, 0, st>>>(n, kn, b0, srb, scb, sb, eb);
    dim3 blk(PT, 8);
    pack_exact_kernel<TA><<<dim3((kn + PT - 1) / PT, (m + PT - 1) / PT, batch), blk, 0, st>>>(
        m, kn, a0, sra, sca, sa, cja, 0, ea, pa, ldo, (long)m * ldo, ldk);
    pack_exact_kernel<TB><<<dim3((kn + PT - 1) / PT, (n + PT - 1) / PT, batch), blk, 0, st>>>(
        n, kn, b0, srb, scb, sb, cjb, 1, eb, pb, ldo, 2L * n * ldo, ldk);
    count_launch(4);
    if (ldk > kr) {
      zero_tails_kernel<<<256, 256, 0, st>>>((long)batch * m, kr, ldk, pa, ldo);
      zero_tails_kernel<<<256, 256, 0, st>>>((long)batch * 2 * n, kr, ldk, pb, ldo);
      count_launch(2);
    }
    MPDO_CUDA_TRY(cudaGetLastError());
    CUtensorMap ma, mb;
    if (!make_map(&ma, 2, pa, ldo, m, ldo, (long)m * ldo, batch, BM) ||
        !make_map(&mb, 2, pb, ldo, 2L * n, ldo, 2L * n * ldo, batch, XBN))
      return cudaErrorInvalidValue;
    dim3 grid((2 * n + XBN - 1) / XBN, (m + BM - 1) / BM, batch);
    const size_t smem = XSTAGES * (BM + XBN) * 128 + 1024 + 256;
    tc_exact_kernel<<<grid, XTHREADS, smem, st>>>(ma, mb, m, 2 * n, kr, ldk, ea, eb,
                                                  reinterpret_cast<double*>(C), 2 * ldc, 2 * sc,
                                                  k0 > 0 ? 1 : 0, err);
    count_launch();
    g_tc_launches.fetch_add(1, std::memory_order_relaxed);
    MPDO_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

cudaError_t tc_pack_real_bf16(cudaStream_t st, int rows, int kc, const float* src, long s_r,
                              long s_c, void* out, long ldo) {
  if (rows <= 0 || kc <= 0) return cudaSuccess;
  dim3 grid((kc + PT - 1) / PT, (rows + PT - 1) / PT), block(PT, 8);
  pack_real_bf16_kernel<<<grid, block, 0, st>>>(rows, kc, src, s_r, s_c,
                                                static_cast<__nv_bfloat16*>(out), ldo);
  count_launch();
  return cudaGetLastError();
}

template cudaError_t tc_cgemm_exact<float2, float2>(cudaStream_t, int, int, int, int, int,
                                                    const float2*, long, long, const float2*,
                                                    long, long, double2*, long, long, int, void*,
                                                    size_t, int*);
template cudaError_t tc_cgemm_exact<float2, double2>(cudaStream_t, int, int, int, int, int,
                                                     const float2*, long, long, const double2*,
                                                     long, long, double2*, long, long, int, void*,
                                                     size_t, int*);
template cudaError_t tc_cgemm_exact<double2, float2>(cudaStream_t, int, int, int, int, int,
                                                     const double2*, long, long, const float2*,
                                                     long, long, double2*, long, long, int, void*,
                                                     size_t, int*);
template cudaError_t tc_cgemm_exact<double2, double2>(cudaStream_t, int, int, int, int, int,
                                                      const double2*, long, long, const double2*,
                                                      long, long, double2*, long, long, int, void*,
                                                      size_t, int*);

size_t tc_cgemm_ws_bytes(int mode, long m, long n, long k, int batch) {
  const int elt = tc_mode_elt(mode);
  const long ld = tc_pack_ld(mode, k);
  return (((size_t)batch * m * ld * elt + 255) & ~(size_t)255) + (size_t)batch * 2 * n * ld * elt;
}

template cudaError_t tc_pack<float>(cudaStream_t, int, int, int, int, const cx<float>*, long, long,
                                    long, int, int, void*);
template cudaError_t tc_pack<double>(cudaStream_t, int, int, int, int, const cx<double>*, long,
                                     long, long, int, int, void*);
template cudaError_t tc_cgemm<float>(cudaStream_t, int, int, int, int, int, int, const cx<float>*,
                                     long, long, const cx<float>*, long, long, float2*, long, long,
                                     int, float2, float2, void*, size_t, int*);

}  // namespace mpdo

// ------------------------------------------------------------------ C ABI (tests)
#include "../../include/mpdo.h"

namespace mpdo {
void set_global_error(const char* msg);
}

namespace {
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};
int tc_fail(int code, const char* msg) {
  mpdo::set_global_error(msg);
  return code;
}
}  // namespace

extern "C" {

long long mpdo_tc_gemm_launches(void) { return mpdo::g_tc_launches.load(); }

int mpdo_kernel_tcgemm_real(int elt, int m, int n, int k, const void* a, long lda, const void* b,
                            long ldb, float* d, long ldd, void* stream) {
  if ((elt != 2 && elt != 4) || m < 0 || n < 0 || k < 1 || !a || !b || !d)
    return tc_fail(MPDO_ERR_ARG, "bad tcgemm_real arguments");
  if ((lda * elt) % 16 || (ldb * elt) % 16 || lda < k || ldb < k || ldd < n)
    return tc_fail(MPDO_ERR_ARG, "tcgemm_real: leading dimensions must cover k (n) and be "
                                 "multiples of 16 bytes");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevBuf err;
  if (cudaMalloc(&err.p, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return tc_fail(MPDO_ERR_OOM, "tcgemm_real: error flag");
  }
  cudaMemsetAsync(err.p, 0, sizeof(int), st);
  mpdo::TcEpilogue e;
  e.d = d;
  e.ldd = ldd;
  cudaError_t ce = mpdo::tc_gemm_real(st, elt, m, n, k, a, lda, 0, b, ldb, 0, 1, e,
                                      static_cast<int*>(err.p), 0);
  int herr = 0;
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return tc_fail(MPDO_ERR_CUDA, cudaGetErrorString(ce));
  if (herr) return tc_fail(MPDO_ERR_TIMEOUT, "tcgemm_real: a pipeline wait gave up");
  return MPDO_OK;
}

int mpdo_kernel_tcgemm(int mode, int opa, int opb, int m, int n, int k, const void* a, long lda,
                       long sa, const void* b, long ldb, long sb, void* c, long ldc, long sc,
                       int batch, void* stream) {
  if (mode < 0 || mode > 3 || opa < 0 || opa > 3 || opb < 0 || opb > 3 || m < 0 || n < 0 ||
      k < 1 || batch < 0 || !a || !b || !c)
    return tc_fail(MPDO_ERR_ARG, "bad tcgemm arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t ws = mpdo::tc_cgemm_ws_bytes(mode, m, n, k, batch);
  DevBuf w, err;
  if (cudaMalloc(&w.p, ws) != cudaSuccess || cudaMalloc(&err.p, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return tc_fail(MPDO_ERR_OOM, "tcgemm workspace");
  }
  cudaMemsetAsync(err.p, 0, sizeof(int), st);
  cudaError_t ce = mpdo::tc_cgemm<float>(
      st, mode, opa, opb, m, n, k, static_cast<const float2*>(a), lda, sa,
      static_cast<const float2*>(b), ldb, sb, static_cast<float2*>(c), ldc, sc, batch,
      make_float2(1.f, 0.f), make_float2(0.f, 0.f), w.p, ws, static_cast<int*>(err.p));
  int herr = 0;
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return tc_fail(MPDO_ERR_CUDA, cudaGetErrorString(ce));
  if (herr) return tc_fail(MPDO_ERR_TIMEOUT, "tcgemm: a pipeline wait gave up");
  return MPDO_OK;
}

int mpdo_kernel_tcgemm_exact(int opa, int opb, int m, int n, int k, const void* a, long lda,
                             long sa, const void* b, long ldb, long sb, void* c, long ldc,
                             long sc, int batch, void* stream) {
  if (opa < 0 || opa > 3 || opb < 0 || opb > 3 || m < 0 || n < 0 || k < 1 || batch < 0 || !a ||
      !b || !c)
    return tc_fail(MPDO_ERR_ARG, "bad tcgemm_exact arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t ws = mpdo::tc_exact_ws_bytes(m, n, k, batch);
  DevBuf w, err;
  if (cudaMalloc(&w.p, ws) != cudaSuccess || cudaMalloc(&err.p, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return tc_fail(MPDO_ERR_OOM, "tcgemm_exact workspace");
  }
  cudaMemsetAsync(err.p, 0, sizeof(int), st);
  cudaError_t ce = mpdo::tc_cgemm_exact<float2, float2>(
      st, opa, opb, m, n, k, static_cast<const float2*>(a), lda, sa, static_cast<const float2*>(b),
      ldb, sb, static_cast<double2*>(c), ldc, sc, batch, w.p, ws, static_cast<int*>(err.p));
  int herr = 0;
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return tc_fail(MPDO_ERR_CUDA, cudaGetErrorString(ce));
  if (herr) return tc_fail(MPDO_ERR_TIMEOUT, "tcgemm_exact: a pipeline wait gave up");
  return MPDO_OK;
}

}  // extern "C"
