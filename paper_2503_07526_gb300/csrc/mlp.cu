// Learned Green-Kubo tail: a fully connected network trained and evaluated
// on the tensor cores (tcgen05.mma with TMEM accumulators, operands staged in
// shared memory by TMA), with FP32 master weights and Adam.
//
// Every product of the forward and backward pass is one launch of k_gemm_tc:
// D [M x N] = A [M x K] * B [N x K]^T with bfloat16 A and B read K-major
// (K contiguous) through 128-byte-swizzled TMA tiles, FP32 accumulation in
// tensor memory, and a fused epilogue (bias, tanh, tanh' from a stored
// activation, output scaling, bfloat16 and FP32 stores, straight or
// transposed).  The transposed stores give the K-major copies that the
// weight-gradient products read (their K is the batch), so no transpose
// kernel runs.
//
// The paper (arXiv 2503.07526) has no learned part; the network, features and
// training are defined in include/gk_tail.h.  Inputs come from the
// multiple-tau readout (Sec. 2.2, Appendix D Algorithm 2); targets are the
// Green-Kubo integrals of Sec. 2.3.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "gk_tail.h"

namespace otf {
namespace tc {

using bf16 = __nv_bfloat16;

constexpr int kBM = 128;     // rows of a CTA tile = MMA M (one TMEM lane per row)
constexpr int kBK = 64;      // K panel: 64 bfloat16 = one 128-byte swizzle row
constexpr int kStages = 2;   // TMA panels in flight
constexpr int kThreads = 128;
constexpr int kOutPad = 16;  // outputs padded to the smallest MMA N
constexpr int kMaxLayers = 8;
constexpr uint64_t kWaitNs = 2000000000ull;  // bounded waits: 2 s of wall time

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity to complete; gives up (false)
// after limit_ns of wall time (at once if the phase is not complete and the
// limit is 0).
__device__ bool mbar_wait_for(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_test(bar, parity)) return true;
  if (limit_ns == 0) return false;
  const uint64_t t0 = global_timer();
  for (;;) {
    if (mbar_test(bar, parity)) return true;
    if (global_timer() - t0 > limit_ns) return false;
    __nanosleep(64);
  }
}
__device__ bool mbar_wait(uint32_t bar, uint32_t parity) { return mbar_wait_for(bar, parity, kWaitNs); }
// 2-D tiled TMA load of box {64 columns, rows} at (x = column, y = row).
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart
// (the stride field); the leading field is unused for this layout.  Bits:
// start address >> 4 at [0,14), leading offset >> 4 at [16,30), stride
// offset >> 4 at [32,46), descriptor version 1 at [46,48), swizzle mode
// (2 = 128 B) at [61,64).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// bfloat16 A and B (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at [17,23), M >> 4 at [24,29).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// Arrives on the barrier once every MMA this thread issued has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Fused epilogue of one product.  x = acc; x += bias[n]; x *= 1 - h^2 with
// h = dact[m][n]; x = tanh(x); x = x * post_scale[n] + post_shift[n]; then
// every non-null output gets x (bfloat16 outputs round to nearest even).
struct Epi {
  const float *bias = nullptr;
  const bf16 *dact = nullptr;
  int64_t ld_dact = 0;
  int act_tanh = 0;
  const float *post_scale = nullptr, *post_shift = nullptr;
  int n_store = 0;     // columns written
  int64_t m_rows = 0;  // rows written
  bf16 *out_b = nullptr;
  int64_t ld_b = 0;
  bf16 *out_bt = nullptr;  // out_bt[n * ld_bt + m]
  int64_t ld_bt = 0;
  float *out_f = nullptr;
  int64_t ld_f = 0;
  float *out_ft = nullptr;  // out_ft[n * ld_ft + m]
  int64_t ld_ft = 0;
};

__host__ __device__ constexpr uint32_t tmem_cols(int N) { return N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256; }
__host__ __device__ constexpr size_t gemm_smem_need(int N) {
  return 1024 + (size_t)kStages * ((size_t)kBM * 128 + (size_t)N * 128) + 64;
}

// One CTA per 128-row tile of D.  Thread 0 issues the TMA loads and the MMAs
// (two panels in flight); all four warps then read their 32 TMEM lanes and
// run the epilogue.  The pipeline waits (a panel landing, a stage's products
// done) give up after wait_ns; the CTA then stops issuing, lets the copies
// it issued land and its products finish (waits of kWaitNs), flags err and
// skips the epilogue, so a stalled pipeline ends as an error status.  K must be a multiple of 16, N a multiple of 16 in
// [16, 256]; rows and columns of A / B past the tensors' ends read as zero.
__global__ void __launch_bounds__(kThreads) k_gemm_tc(const __grid_constant__ CUtensorMap ta,
                                                      const __grid_constant__ CUtensorMap tb, int K, int N,
                                                      int a_row0, int a_k0, int b_row0, int b_k0, Epi e,
                                                      unsigned *err, uint64_t wait_ns) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const uint32_t a_bytes = kBM * 128, b_bytes = (uint32_t)N * 128;
  uint8_t *sa = smem;
  uint8_t *sb = smem + kStages * a_bytes;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sb + kStages * b_bytes);  // full[S], empty[S], done
  uint32_t *slot = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 1);
  int *flag = reinterpret_cast<int *>(slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t ncols = tmem_cols(N);
  const uint32_t done_bar = smem_u32(&bars[2 * kStages]);

  if (tid == 0) {
    for (int s = 0; s < 2 * kStages + 1; ++s) mbar_init(smem_u32(&bars[s]), 1);
    *flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(slot), ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const int m0 = blockIdx.x * kBM;

  if (tid == 0) {
    const int np = (K + kBK - 1) / kBK;
    const uint32_t idesc = idesc_bf16(kBM, N);
    int issued = 0, consumed = 0;
    bool ok = true;
    auto load = [&](int p, int s) {
      const uint32_t fb = smem_u32(&bars[s]);
      mbar_expect_tx(fb, a_bytes + b_bytes);
      tma_load_2d(smem_u32(sa + s * a_bytes), &ta, a_k0 + p * kBK, a_row0 + m0, fb);
      tma_load_2d(smem_u32(sb + s * b_bytes), &tb, b_k0 + p * kBK, b_row0, fb);
      ++issued;
    };
    for (int p = 0; p < np && p < kStages; ++p) load(p, p);
    for (int p = 0; p < np; ++p) {
      const int s = p % kStages;
      const uint32_t ph = (uint32_t)(p / kStages) & 1u;
      if (!mbar_wait_for(smem_u32(&bars[s]), ph, wait_ns)) {
        ok = false;
        break;
      }
      ++consumed;
      tc_fence_after();
      const int nk = min(kBK, K - p * kBK) / 16;
      const uint32_t a0 = smem_u32(sa + s * a_bytes), b0 = smem_u32(sb + s * b_bytes);
      for (int j = 0; j < nk; ++j)
        mma_bf16(tmem, sw128_desc(a0 + 32u * j), sw128_desc(b0 + 32u * j), idesc, (p | j) != 0);
      mma_commit(smem_u32(&bars[kStages + s]));
      if (p + kStages < np) {
        if (!mbar_wait_for(smem_u32(&bars[kStages + s]), ph, wait_ns)) {
          ok = false;
          break;
        }
        load(p + kStages, s);
      }
    }
    mma_commit(done_bar);
    if (!ok) {
      // let the copies already issued land before the CTA exits
      for (int p = consumed; p < issued; ++p) mbar_wait(smem_u32(&bars[p % kStages]), (uint32_t)(p / kStages) & 1u);
      *flag = 1;
    }
  }
  const bool done_ok = mbar_wait(done_bar, 0);
  tc_fence_after();
  __syncthreads();
  const bool run = done_ok && *flag == 0;
  if (!run && tid == 0) atomicOr(err, 1u);

  // bfloat16 row-major output: staged through the (now idle) operand
  // buffers and written row by row with 16-byte stores, so a warp writes
  // whole lines (a thread owns a row of the accumulator, so direct stores
  // would touch 32 rows per instruction)
  const bool stage_b = e.out_b && e.n_store == N && N % 8 == 0 && e.ld_b % 8 == 0 &&
                       (reinterpret_cast<uintptr_t>(e.out_b) & 15) == 0;
  const int pitch = N + 8;  // staged row, in bfloat16
  bf16 *stile = reinterpret_cast<bf16 *>(smem);
  if (run) {
    const int row = warp * 32 + lane;
    const int64_t m = (int64_t)m0 + row;
    const bool live = m < e.m_rows;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tmem_ld16(trow + (uint32_t)c0, v);  // warp-collective: every lane loads
      if (!live) continue;
      float hd[16];
      if (e.dact) {  // the 16 stored activations of this row and column group
        const bf16 *hp = e.dact + m * e.ld_dact + c0;
        if ((e.ld_dact % 8) == 0 && (reinterpret_cast<uintptr_t>(e.dact) & 15) == 0 && c0 + 16 <= e.n_store) {
          const uint4 q0 = *reinterpret_cast<const uint4 *>(hp), q1 = *reinterpret_cast<const uint4 *>(hp + 8);
          const bf16 *b0 = reinterpret_cast<const bf16 *>(&q0), *b1 = reinterpret_cast<const bf16 *>(&q1);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            hd[i] = __bfloat162float(b0[i]);
            hd[8 + i] = __bfloat162float(b1[i]);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) hd[i] = c0 + i < e.n_store ? __bfloat162float(hp[i]) : 0.f;
        }
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int n = c0 + i;
        if (n >= e.n_store) break;
        float x = v[i];
        if (e.bias) x += e.bias[n];
        if (e.dact) x *= 1.0f - hd[i] * hd[i];
        if (e.act_tanh) x = tanhf(x);
        if (e.post_scale) x = fmaf(x, e.post_scale[n], e.post_shift[n]);
        if (e.out_f) e.out_f[m * e.ld_f + n] = x;
        if (e.out_ft) e.out_ft[(int64_t)n * e.ld_ft + m] = x;
        const bf16 xb = __float2bfloat16_rn(x);
        if (stage_b)
          stile[row * pitch + n] = xb;
        else if (e.out_b)
          e.out_b[m * e.ld_b + n] = xb;
        if (e.out_bt) e.out_bt[(int64_t)n * e.ld_bt + m] = xb;
      }
    }
  }
  if (stage_b) {
    __syncthreads();
    if (run) {
      const int per_row = N / 8;
      for (int k = tid; k < kBM * per_row; k += kThreads) {
        const int row = k / per_row, c8 = k % per_row;
        const int64_t m = (int64_t)m0 + row;
        if (m < e.m_rows)
          *reinterpret_cast<uint4 *>(e.out_b + m * e.ld_b + c8 * 8) =
              *reinterpret_cast<const uint4 *>(stile + row * pitch + c8 * 8);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// ------------------------------------------------- fused inference forward
//
// The whole forward pass of a 128-row tile in one CTA: every layer's weights
// stay in shared memory (loaded once per CTA by TMA), the inputs are
// standardised and rounded to bfloat16 on the way into shared memory, and
// each hidden layer's activations go from TMEM through the epilogue straight
// back into shared memory as the next product's A operand, so only the
// FP32 inputs and outputs cross HBM.  A CTA runs two groups of eight warps,
// each group on its own tile (its own activation buffer and 128 TMEM
// columns; two warps share each 32-lane quarter of TMEM and split its
// columns), so one group's epilogue overlaps the other's tensor-core
// products; the CTA is persistent over tiles.  Rounding points are those of
// the layered path (bfloat16 inputs, weights and activations, FP32
// accumulation); the inputs are standardised with the FP32 reciprocal of the
// scale (within two FP32 units of the quotient) and tanh is evaluated as in
// tanh2_epi below.
constexpr int kFusedGroup = 256;                   // threads of a group: eight warps, one tile
constexpr int kFusedThreads = 2 * kFusedGroup;     // two groups
constexpr int kInBatch = 3;  // input units (8 columns of a row) whose loads a thread has in flight at once
constexpr uint32_t kPanelBytes = kBM * 128;        // 128 rows x 64 bfloat16

struct FusedMaps {
  CUtensorMap w[kMaxLayers];  // W_l [out_p][in_k] bfloat16, boxes {64, out_p}
};
struct FusedArgs {
  int L = 0, n_in = 0, k_in = 0, n_out = 0, unscale = 0;
  int in_k[kMaxLayers] = {}, out_p[kMaxLayers] = {};
  uint32_t w_off[kMaxLayers] = {};  // byte offset of layer l's panels in shared memory
  uint32_t w_bytes = 0, act_bytes = 0;
  int b_off[kMaxLayers] = {};       // offset of layer l's bias in the shared bias table
  int nbias = 0;                    // a multiple of 16
  const float *bias[kMaxLayers] = {};
  const float *xmean = nullptr, *xstd = nullptr, *ymean = nullptr, *ystd = nullptr;
};

// Paired FP32 arithmetic (two lanes of a 64-bit register, each rounded to
// nearest like the scalar instruction) for the epilogue.
__device__ __forceinline__ uint64_t f2_pack(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t r, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// tanh of two pre-activations z = acc + bias for the epilogue, as
// 1 - 2 / (exp(2z) + 1) from the hardware base-2 exponential and reciprocal.
// The result tends to +-1 with the right sign as exp(2z) overflows or
// underflows; its absolute error is about 2e-7 everywhere, below the
// bfloat16 rounding of every activation larger than 1e-4 in magnitude that
// follows (smaller ones are off by at most that 2e-7, which no normwise
// comparison can see).
__device__ __forceinline__ uint64_t tanh2_epi(uint64_t acc, uint64_t bias) {
  const uint64_t y = f2_mul(f2_add(acc, bias), f2_pack(2.8853900817779268f, 2.8853900817779268f));  // 2 log2(e) z
  float y0, y1, e0, e1, r0, r1;
  f2_unpack(y, y0, y1);
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e0) : "f"(y0));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(y1));
  const uint64_t d = f2_add(f2_pack(e0, e1), f2_pack(1.0f, 1.0f));
  f2_unpack(d, e0, e1);
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(e0));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(e1));
  return f2_fma(f2_pack(-2.0f, -2.0f), f2_pack(r0, r1), f2_pack(1.0f, 1.0f));
}

// Waits on a phase of an mbarrier with the potentially blocking try_wait
// (the thread is suspended in hardware rather than spinning); gives up
// (false) after kWaitNs.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ bool mbar_wait_blocking(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_timer();
  while (!mbar_try(bar, parity))
    if (global_timer() - t0 > kWaitNs) return false;
  return true;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void group_sync(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kFusedGroup) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Eight values as bfloat16 into 16-byte chunk `ch` of row `r` of a K-major
// operand tile laid out as a 128-byte-swizzled TMA load would leave it:
// 64-column panels of 128 rows x 128 bytes, chunk j of row r at
// r * 128 + ((j ^ (r mod 8)) * 16) within its panel.
__device__ __forceinline__ void store_chunk_sw128(uint8_t *tile, int r, int ch, const float (&x)[8]) {
  uint4 q;
  __nv_bfloat162 b0 = __floats2bfloat162_rn(x[0], x[1]), b1 = __floats2bfloat162_rn(x[2], x[3]);
  __nv_bfloat162 b2 = __floats2bfloat162_rn(x[4], x[5]), b3 = __floats2bfloat162_rn(x[6], x[7]);
  q.x = *reinterpret_cast<uint32_t *>(&b0);
  q.y = *reinterpret_cast<uint32_t *>(&b1);
  q.z = *reinterpret_cast<uint32_t *>(&b2);
  q.w = *reinterpret_cast<uint32_t *>(&b3);
  const int p = ch >> 3, j = ch & 7;
  *reinterpret_cast<uint4 *>(tile + (size_t)p * kPanelBytes + r * 128 + ((j ^ (r & 7)) << 4)) = q;
}

// Shared tables after the activation tiles: biases [nbias], input means and
// reciprocal scales [k_in] each (zero past n_in), output scale and shift
// [16] each; then the barriers.
__host__ __device__ constexpr size_t fused_tables_bytes(int nbias, int k_in) {
  return sizeof(float) * ((size_t)nbias + 2 * (size_t)k_in + 2 * kOutPad) + 64;
}

__global__ void __launch_bounds__(kFusedThreads, 1)
    k_mlp_fused(const __grid_constant__ FusedMaps maps, const FusedArgs a, const float *__restrict__ X,
                int64_t rows, float *__restrict__ Y, unsigned *err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t *sw = smem;
  uint8_t *sact = smem + a.w_bytes;
  float *sbias = reinterpret_cast<float *>(sact + 2 * (size_t)a.act_bytes);
  float *sxm = sbias + a.nbias, *sxr = sxm + a.k_in, *sym = sxr + a.k_in, *sys = sym + kOutPad;
  uint64_t *bars = reinterpret_cast<uint64_t *>((reinterpret_cast<uintptr_t>(sys + kOutPad) + 7) & ~(uintptr_t)7);
  // bars: weights, group 0 MMA, group 1 MMA, group 0 inputs done, group 1 inputs done
  uint32_t *slot = reinterpret_cast<uint32_t *>(bars + 5);
  int *gflag = reinterpret_cast<int *>(slot + 1);            // [2]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = tid / kFusedGroup, gt = tid % kFusedGroup, gw = warp & 7;
  const int quarter = gw & 3, half = gw >> 2;  // TMEM lane quarter, column half of the warp
  const uint32_t wbar = smem_u32(&bars[0]);

  if (tid == 0) {
    for (int s = 0; s < 5; ++s) mbar_init(smem_u32(&bars[s]), 1);
    gflag[0] = gflag[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(slot), 256);
  for (int l = 0; l < a.L; ++l)
    for (int c = tid; c < a.out_p[l]; c += kFusedThreads) sbias[a.b_off[l] + c] = a.bias[l][c];
  for (int c = tid; c < a.k_in; c += kFusedThreads) {
    sxm[c] = c < a.n_in ? a.xmean[c] : 0.f;
    sxr[c] = c < a.n_in ? 1.0f / a.xstd[c] : 0.f;
  }
  for (int c = tid; c < kOutPad; c += kFusedThreads) {
    sym[c] = a.unscale ? a.ymean[c] : 0.f;
    sys[c] = a.unscale ? a.ystd[c] : 1.f;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  if (tid == 0) {  // every layer's weight panels, one transaction
    mbar_expect_tx(wbar, a.w_bytes);
    for (int l = 0; l < a.L; ++l) {
      const uint32_t pb = (uint32_t)a.out_p[l] * 128u;
      for (int p = 0; p * kBK < a.in_k[l]; ++p)
        tma_load_2d(smem_u32(sw + a.w_off[l] + p * pb), &maps.w[l], p * kBK, 0, wbar);
    }
  }

  uint8_t *act = sact + (size_t)g * a.act_bytes;
  const uint32_t act_s = smem_u32(act);
  const uint32_t mbar = smem_u32(&bars[1 + g]);
  const uint32_t dcol = tmem + (uint32_t)(g * 128);                                 // the group's accumulator
  const uint32_t trow = dcol + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 64);  // this warp's part
  const int row = quarter * 32 + lane;                                              // tile row = TMEM lane
  const int nch = a.k_in / 8;
  const int r0 = gt / nch, ch0 = gt % nch, dr = kFusedGroup / nch, dch = kFusedGroup % nch;
  const bool vec = (a.n_in % 4) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  uint32_t phase = 0;
  bool have_w = false;
  const int64_t ntiles = (rows + kBM - 1) / kBM;
  // The two groups take turns at their input stages (group 0's k-th, then
  // group 1's k-th, then group 0's (k+1)-th, ...), so one group streams its
  // inputs while the other runs products and epilogues instead of both
  // doing the same phase at the same time.  A group's tile count is at most
  // one more than the other's, so every wait below has its arrival.
  int k = 0;
  for (int64_t t = 2 * (int64_t)blockIdx.x + g; t < ntiles && !gflag[g]; t += 2 * (int64_t)gridDim.x, ++k) {
    const int64_t m0 = t * kBM;
    if (g == 1 || k > 0) {
      const int other = 1 - g, kk = g == 1 ? k : k - 1;  // the other group's input stage to follow
      if (!mbar_wait_blocking(smem_u32(&bars[3 + other]), (uint32_t)kk & 1u)) gflag[g] = 1;
    }
    // inputs: standardised, rounded to bfloat16, swizzled into the A tile;
    // unit (r, ch) is eight columns of row r
    int r = r0, ch = ch0;
    const int units = kBM * nch;
    for (int u0 = gt; u0 < units; u0 += kInBatch * kFusedGroup) {
      // kInBatch units' loads in flight before any of them is used
      float x[kInBatch][8];
      int rr[kInBatch], cc[kInBatch];
#pragma unroll
      for (int k = 0; k < kInBatch; ++k) {
        rr[k] = r;
        cc[k] = ch;
        const int64_t m = m0 + r;
        const int c0 = ch * 8;
        if (u0 + k * kFusedGroup < units && m < rows && vec && c0 + 8 <= a.n_in) {
          const float4 p0 = __ldcs(reinterpret_cast<const float4 *>(X + m * a.n_in + c0));
          const float4 p1 = __ldcs(reinterpret_cast<const float4 *>(X + m * a.n_in + c0 + 4));
          x[k][0] = p0.x, x[k][1] = p0.y, x[k][2] = p0.z, x[k][3] = p0.w;
          x[k][4] = p1.x, x[k][5] = p1.y, x[k][6] = p1.z, x[k][7] = p1.w;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            x[k][e] = (u0 + k * kFusedGroup < units && m < rows && c0 + e < a.n_in) ? X[m * a.n_in + c0 + e] : 0.f;
        }
        r += dr;
        ch += dch;
        if (ch >= nch) {
          ch -= nch;
          ++r;
        }
      }
#pragma unroll
      for (int k = 0; k < kInBatch; ++k) {
        if (u0 + k * kFusedGroup >= units) break;
        const int c0 = cc[k] * 8;
        const float4 mu0 = *reinterpret_cast<const float4 *>(sxm + c0);
        const float4 mu1 = *reinterpret_cast<const float4 *>(sxm + c0 + 4);
        const float4 rs0 = *reinterpret_cast<const float4 *>(sxr + c0);
        const float4 rs1 = *reinterpret_cast<const float4 *>(sxr + c0 + 4);
        float y[8] = {(x[k][0] - mu0.x) * rs0.x, (x[k][1] - mu0.y) * rs0.y, (x[k][2] - mu0.z) * rs0.z,
                      (x[k][3] - mu0.w) * rs0.w, (x[k][4] - mu1.x) * rs1.x, (x[k][5] - mu1.y) * rs1.y,
                      (x[k][6] - mu1.z) * rs1.z, (x[k][7] - mu1.w) * rs1.w};
        store_chunk_sw128(act, rr[k], cc[k], y);
      }
    }
    fence_proxy_async();
    group_sync(1 + g);
    if (gt == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bars[3 + g])) : "memory");
    if (gflag[g]) break;
    // the group's next tile's inputs (one contiguous block) on their way
    // into L2 while this tile's products and epilogues run
    const int64_t mn = m0 + 2 * (int64_t)gridDim.x * kBM;
    if (gt == 0 && vec && mn < rows) {
      const uint32_t bytes = (uint32_t)(min((int64_t)kBM, rows - mn) * a.n_in * (int64_t)sizeof(float));
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(X + mn * a.n_in), "r"(bytes) : "memory");
    }
    for (int l = 0; l < a.L; ++l) {
      if (gt == 0) {
        const bool ok = have_w || mbar_wait_blocking(wbar, 0);
        have_w = ok;
        tc_fence_after();
        if (ok) {
          const uint32_t idesc = idesc_bf16(kBM, a.out_p[l]);
          const uint32_t wb = smem_u32(sw + a.w_off[l]), pb = (uint32_t)a.out_p[l] * 128u;
          for (int kk = 0; kk < a.in_k[l] / 16; ++kk) {
            const int p = kk >> 2, j = kk & 3;
            mma_bf16(dcol, sw128_desc(act_s + p * kPanelBytes + 32u * j), sw128_desc(wb + p * pb + 32u * j), idesc,
                     kk > 0);
          }
        } else {
          gflag[g] = 1;
        }
        mma_commit(mbar);  // arrives once the products (if any) are done
      }
      const bool done = __all_sync(0xffffffffu, mbar_wait_blocking(mbar, phase));
      phase ^= 1u;
      tc_fence_after();
      if (!done) {
        gflag[g] = 1;
      } else if (l < a.L - 1) {
        // bias, tanh, bfloat16 of this warp's 32 rows x 64 columns: the next
        // product's A tile
        const float *bl = sbias + a.b_off[l] + half * 64;
#pragma unroll 1
        for (int c0 = 0; c0 < 64; c0 += 32) {
          float v[32];
          tmem_ld32(trow + (uint32_t)c0, v);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float x[8];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
              const int c = c0 + q * 8 + e;
              const float2 b2 = *reinterpret_cast<const float2 *>(bl + c);
              f2_unpack(tanh2_epi(f2_pack(v[q * 8 + e], v[q * 8 + e + 1]), f2_pack(b2.x, b2.y)), x[e], x[e + 1]);
            }
            store_chunk_sw128(act, row, half * 8 + c0 / 8 + q, x);
          }
        }
      } else if (half == 0) {
        float v[16];
        tmem_ld16(trow, v);
        const int64_t m = m0 + row;
        if (m < rows) {
          const float *bl = sbias + a.b_off[l];
#pragma unroll
          for (int c = 0; c < kOutPad; ++c)
            if (c < a.n_out) Y[m * a.n_out + c] = fmaf(v[c] + bl[c], sys[c], sym[c]);
        }
      }
      tc_fence_before();
      fence_proxy_async();
      group_sync(1 + g);
      if (gflag[g]) break;
    }
  }
  if (tid == 0) mbar_wait(wbar, 0);  // the weight copies have landed before the CTA can exit
  if (gt == 0 && gflag[g]) atomicOr(err, 1u);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

// Standardised, bfloat16-rounded inputs: out [rows_pad][k] row-major and
// (optional) out_t [k][ld_t]; pad columns and rows past `rows` are zero.
__global__ void k_prep_x(const float *__restrict__ X, int64_t rows, int n_in, const float *__restrict__ mean,
                         const float *__restrict__ stdv, bf16 *__restrict__ out, int64_t rows_pad, int k,
                         bf16 *__restrict__ out_t, int64_t ld_t) {
  const int64_t total = rows_pad * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = i / k;
    const int c = (int)(i % k);
    float x = 0.f;
    if (m < rows && c < n_in) x = (X[m * n_in + c] - mean[c]) / stdv[c];
    const bf16 xb = __float2bfloat16_rn(x);
    out[i] = xb;
    if (out_t) out_t[(int64_t)c * ld_t + m] = xb;
  }
}

// Standardised targets.
__global__ void k_prep_t(const float *__restrict__ T, int64_t rows, int n_out, const float *__restrict__ mean,
                         const float *__restrict__ stdv, float *__restrict__ out) {
  const int64_t total = rows * n_out;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % n_out);
    out[i] = (T[i] - mean[c]) / stdv[c];
  }
}

// One epoch's sample order: rows of the prepared inputs and targets gathered
// into X [n][k], its transpose [k][n], and T [n][n_out].
__global__ void k_gather(const bf16 *__restrict__ Xall, const float *__restrict__ Tall, const int64_t *__restrict__ perm,
                         int64_t n, int k, int n_out, bf16 *__restrict__ Xs, bf16 *__restrict__ Xst,
                         float *__restrict__ Ts) {
  const int64_t total = n * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = i / k;
    const int c = (int)(i % k);
    const int64_t src = perm[m];
    const bf16 x = Xall[src * k + c];
    Xs[i] = x;
    Xst[(int64_t)c * n + m] = x;
    if (c < n_out) Ts[m * n_out + c] = Tall[src * n_out + c];
  }
}

// Loss of one batch and the output gradient dY = 2 (y - t) / (rows n_out),
// bfloat16, into dY [rows][64] and dYt [16][ld_t] (pads stay zero).  One
// block; the sum runs in a fixed order, so the loss is reproducible.
// loss_acc[0] += loss * acc_scale; loss_acc[1] = loss.
__global__ void k_loss_dy(const float *__restrict__ Y, const float *__restrict__ T, int64_t rows, int n_out,
                          bf16 *__restrict__ dY, bf16 *__restrict__ dYt, int64_t ld_t, double *loss_acc,
                          double acc_scale) {
  __shared__ double part[256];
  const double inv = 1.0 / ((double)rows * n_out);
  const float g = (float)(2.0 * inv);
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < rows * n_out; i += blockDim.x) {
    const int64_t m = i / n_out;
    const int c = (int)(i % n_out);
    const float d = Y[m * kOutPad + c] - T[i];
    acc += (double)d * d;
    const bf16 db = __float2bfloat16_rn(g * d);
    dY[m * 64 + c] = db;
    dYt[(int64_t)c * ld_t + m] = db;
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double L = part[0] * inv;
    loss_acc[0] += L * acc_scale;
    loss_acc[1] = L;
  }
}

// Bias gradients: dst_l[n] = sum over m < rows of src_l[n][m] (bfloat16 dZ^T
// rows), one warp per (layer, n), fixed summation order.
struct BiasJob {
  const bf16 *src;
  int64_t ld;
  float *dst;
  int count;
};
struct BiasJobs {
  BiasJob j[kMaxLayers];
  int n;
};
__global__ void k_bias_grad(BiasJobs jobs, int64_t rows) {
  const BiasJob &J = jobs.j[blockIdx.y];
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= J.count) return;
  const bf16 *s = J.src + (int64_t)w * J.ld;
  float acc = 0.f;
  for (int64_t m = lane; m < rows; m += 32) acc += __bfloat162float(s[m]);
  acc = warp_sum(acc);
  if (lane == 0) J.dst[w] = acc;
}

// Adam with bias correction (c1 = 1 - beta1^t, c2 = 1 - beta2^t) and
// decoupled weight decay on weight matrices, over the padded parameter
// vector; refreshes the bfloat16 copies W [out_p][in_k] and (when present)
// W^T [in_k][ld_t].
struct AdamLayer {
  int64_t w_off, b_off;
  int out_p, in_k;
  bf16 *wb, *wtb;
  int ld_t;
};
struct AdamTable {
  AdamLayer l[kMaxLayers];
  int n;
};
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, int64_t count, AdamTable tab, float lr, float beta1, float beta2,
                       float eps, float wd, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    int L = 0;
    bool is_w = false;
    for (int l = 0; l < tab.n; ++l) {
      const AdamLayer &A = tab.l[l];
      if (i >= A.w_off && i < A.w_off + (int64_t)A.out_p * A.in_k) {
        L = l;
        is_w = true;
      }
      if (i >= A.b_off && i < A.b_off + A.out_p) L = l;
    }
    const float gi = g[i];
    const float a = beta1 * m1[i] + (1.f - beta1) * gi;
    const float b = beta2 * m2[i] + (1.f - beta2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    float step = (a / c1) / (sqrtf(b / c2) + eps);
    if (is_w) step += wd * w[i];
    const float wn = w[i] - lr * step;
    w[i] = wn;
    if (is_w) {
      const AdamLayer &A = tab.l[L];
      const int64_t j = i - A.w_off;
      const int o = (int)(j / A.in_k), c = (int)(j % A.in_k);
      const bf16 wbv = __float2bfloat16_rn(wn);
      A.wb[j] = wbv;
      if (A.wtb) A.wtb[(int64_t)c * A.ld_t + o] = wbv;
    }
  }
}

// bfloat16 copies of the master weights (after set / init).
__global__ void k_cast_weights(const float *__restrict__ w, AdamTable tab) {
  const AdamLayer &A = tab.l[blockIdx.y];
  const int64_t n = (int64_t)A.out_p * A.in_k;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int o = (int)(j / A.in_k), c = (int)(j % A.in_k);
    const bf16 v = __float2bfloat16_rn(w[A.w_off + j]);
    A.wb[j] = v;
    if (A.wtb) A.wtb[(int64_t)c * A.ld_t + o] = v;
  }
}

// ---------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map of a row-major bfloat16 matrix [outer][inner], read in boxes of
// 64 columns x box_rows rows with 128-byte swizzle.
int make_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return MD_ECUDA;
  }
  if (inner % 8 || inner < 64 || box_rows < 1 || box_rows > 256) {
    set_error("tensor map: inner extent %llu / box rows %u not supported", (unsigned long long)inner, box_rows);
    return MD_EINVAL;
  }
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * sizeof(bf16)};
  cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return MD_ECUDA;
  }
  return MD_OK;
}

struct Mat {  // a bfloat16 device matrix with its tensor map
  bf16 *p = nullptr;
  int64_t rows = 0, cols = 0;
  CUtensorMap map;  // the type carries the alignment the driver needs
};

int mat_alloc(Mat &M, int64_t rows, int64_t cols, uint32_t box_rows) {
  M.rows = rows;
  M.cols = cols;
  OTF_CUDA(cudaMalloc(&M.p, sizeof(bf16) * rows * cols));
  OTF_CUDA(cudaMemset(M.p, 0, sizeof(bf16) * rows * cols));
  return make_map(&M.map, M.p, (uint64_t)cols, (uint64_t)rows, box_rows);
}
void mat_free(Mat &M) {
  if (M.p) cudaFree(M.p);
  M.p = nullptr;
}

int launch_gemm(cudaStream_t st, const Mat &A, int a_row0, int a_k0, const Mat &B, int b_row0, int b_k0, int64_t M,
                int N, int K, const Epi &e, unsigned *err, uint64_t wait_ns) {
  if (N % 16 || N < 16 || N > 256 || K % 16 || K < 16) {
    set_error("k_gemm_tc: N = %d, K = %d not supported", N, K);
    return MD_EINVAL;
  }
  size_t smem = gemm_smem_need(N);
  // at most two CTAs of 256 TMEM columns per SM (512 columns in all)
  if (tmem_cols(N) == 256) smem = std::max<size_t>(smem, 80 * 1024);
  static std::once_flag once;
  static cudaError_t attr_rc = cudaSuccess;
  std::call_once(once, [] {
    attr_rc = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  });
  OTF_CUDA(attr_rc);
  const int grid = ceil_div(M, kBM);
  k_gemm_tc<<<grid, kThreads, smem, st>>>(A.map, B.map, K, N, a_row0, a_k0, b_row0, b_k0, e, err, wait_ns);
  OTF_LAUNCH_CHECK();
  return MD_OK;
}

// SplitMix64 (Steele, Lea and Flood 2014): output k (k >= 1) of the stream
// with the given seed, and a uniform double in [0, 1) from its top 53 bits.
uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uniform01_at(uint64_t seed, uint64_t k) { return (double)(splitmix64_at(seed, k) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace tc
}  // namespace otf

using namespace otf;
using namespace otf::tc;

struct mlp_handle_s {
  cudaStream_t st = nullptr;
  uint64_t wait_ns = kWaitNs;  // limit of the tensor-core pipeline waits (mlp_set_wait_limit)
  mlp_params p{};
  int L = 0;          // layers = depth + 1
  int k_in = 0;       // padded input width
  int cap = 0;        // training batch rows
  struct Layer {
    int in = 0, out = 0, in_k = 0, out_p = 0;
    int64_t w_off = 0, b_off = 0;  // into the padded parameter vector
    Mat wb, wtb;                   // bfloat16 W [out_p][in_k], W^T [in_k][out_p or 64]
  };
  std::vector<Layer> lay;
  int64_t np_pad = 0, np_flat = 0;
  float *w = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
  int64_t t = 0;  // Adam steps taken
  float *xmean = nullptr, *xstd = nullptr, *ymean = nullptr, *ystd = nullptr;  // device scaler
  std::vector<float> h_xmean, h_xstd, h_ymean, h_ystd;
  // training batch state
  Mat xb, xbt;              // [cap][k_in], [k_in][cap]
  std::vector<Mat> H, Ht;   // per hidden layer: [cap][width], [width][cap]
  std::vector<Mat> dZ, dZt; // per hidden layer
  Mat dY, dYt;              // [cap][64], [16][cap]
  float *Y = nullptr;       // [cap][16]
  float *T = nullptr;       // [cap][n_out]
  double *loss = nullptr;   // [2]
  unsigned *err = nullptr;
  unsigned *err_host = nullptr;  // pinned copy of err, read after each call
  // inference state (grown on demand)
  int64_t icap = 0;
  Mat xi;
  Mat hi[2];
  float *Yi = nullptr;
  AdamTable table{};
  // fused inference forward (when every layer's weights and two activation
  // tiles fit in one CTA's shared memory)
  bool fused = false;
  size_t fused_smem = 0;
  int nsm = 0;
  FusedArgs fa{};
  FusedMaps fm;
};

namespace {

int check_err(mlp_handle *h) {
  OTF_CUDA(cudaMemcpyAsync(h->err_host, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->st));
  OTF_CUDA(cudaStreamSynchronize(h->st));
  const unsigned e = *h->err_host;
  if (e) {
    cudaMemsetAsync(h->err, 0, sizeof(unsigned), h->st);
    set_error("a bounded tensor-core pipeline wait gave up");
    return MD_ETIMEOUT;
  }
  return MD_OK;
}

int upload_scaler(mlp_handle *h) {
  std::vector<float> ym(kOutPad, 0.f), ys(kOutPad, 1.f);
  std::copy(h->h_ymean.begin(), h->h_ymean.end(), ym.begin());
  std::copy(h->h_ystd.begin(), h->h_ystd.end(), ys.begin());
  OTF_CUDA(cudaMemcpyAsync(h->xmean, h->h_xmean.data(), sizeof(float) * h->p.n_in, cudaMemcpyHostToDevice, h->st));
  OTF_CUDA(cudaMemcpyAsync(h->xstd, h->h_xstd.data(), sizeof(float) * h->p.n_in, cudaMemcpyHostToDevice, h->st));
  OTF_CUDA(cudaMemcpyAsync(h->ymean, ym.data(), sizeof(float) * kOutPad, cudaMemcpyHostToDevice, h->st));
  OTF_CUDA(cudaMemcpyAsync(h->ystd, ys.data(), sizeof(float) * kOutPad, cudaMemcpyHostToDevice, h->st));
  OTF_CUDA(cudaStreamSynchronize(h->st));
  return MD_OK;
}

int cast_weights(mlp_handle *h) {
  dim3 grid(64, h->L);
  k_cast_weights<<<grid, 256, 0, h->st>>>(h->w, h->table);
  OTF_LAUNCH_CHECK();
  return MD_OK;
}

// flat (unpadded, API order) <-> padded device layout, on the host
void flat_to_pad(const mlp_handle *h, const float *flat, std::vector<float> &pad) {
  pad.assign((size_t)h->np_pad, 0.f);
  int64_t f = 0;
  for (const auto &Ly : h->lay) {
    for (int o = 0; o < Ly.out; ++o)
      for (int i = 0; i < Ly.in; ++i) pad[(size_t)(Ly.w_off + (int64_t)o * Ly.in_k + i)] = flat[f++];
    for (int o = 0; o < Ly.out; ++o) pad[(size_t)(Ly.b_off + o)] = flat[f++];
  }
}
void pad_to_flat(const mlp_handle *h, const std::vector<float> &pad, float *flat) {
  int64_t f = 0;
  for (const auto &Ly : h->lay) {
    for (int o = 0; o < Ly.out; ++o)
      for (int i = 0; i < Ly.in; ++i) flat[f++] = pad[(size_t)(Ly.w_off + (int64_t)o * Ly.in_k + i)];
    for (int o = 0; o < Ly.out; ++o) flat[f++] = pad[(size_t)(Ly.b_off + o)];
  }
}

int reset_adam(mlp_handle *h) {
  OTF_CUDA(cudaMemsetAsync(h->m1, 0, sizeof(float) * h->np_pad, h->st));
  OTF_CUDA(cudaMemsetAsync(h->m2, 0, sizeof(float) * h->np_pad, h->st));
  h->t = 0;
  return MD_OK;
}

// Forward pass of `rows` rows whose prepared inputs are rows [row0, row0+rows)
// of X.  Hidden activations go to Hs (ping-pong when Hs has 2 entries and no
// transposes are kept), the output to Y [.][16].
int forward(mlp_handle *h, const Mat &X, int row0, int64_t rows, Mat *Hs, int nH, Mat *Hts, float *Y,
            bool unscale) {
  const int L = h->L;
  for (int l = 0; l < L; ++l) {
    const auto &Ly = h->lay[l];
    const Mat &A = (l == 0) ? X : Hs[(l - 1) % nH];
    Epi e;
    e.bias = h->w + Ly.b_off;
    e.m_rows = rows;
    if (l < L - 1) {
      Mat &out = Hs[l % nH];
      e.act_tanh = 1;
      e.n_store = Ly.out_p;
      e.out_b = out.p;
      e.ld_b = out.cols;
      if (Hts) {
        e.out_bt = Hts[l].p;
        e.ld_bt = Hts[l].cols;
      }
    } else {
      e.n_store = kOutPad;
      e.out_f = Y;
      e.ld_f = kOutPad;
      if (unscale) {
        e.post_scale = h->ystd;
        e.post_shift = h->ymean;
      }
    }
    int rc = launch_gemm(h->st, A, l == 0 ? row0 : 0, 0, Ly.wb, 0, 0, rows, Ly.out_p, Ly.in_k, e, h->err, h->wait_ns);
    if (rc) return rc;
  }
  return MD_OK;
}

// Forward + backward on one batch: inputs rows [row0, row0+cap) of X (with
// its transpose Xt, K offset row0), standardised targets Tb [cap][n_out].
// Gradients land in h->g (padded layout).
int train_step(mlp_handle *h, const Mat &X, const Mat &Xt, int row0, const float *Tb, double acc_scale) {
  const int L = h->L, cap = h->cap;
  int rc = forward(h, X, row0, cap, h->H.data(), (int)h->H.size(), h->Ht.data(), h->Y, false);
  if (rc) return rc;
  k_loss_dy<<<1, 256, 0, h->st>>>(h->Y, Tb, cap, h->p.n_out, h->dY.p, h->dYt.p, cap, h->loss, acc_scale);
  OTF_LAUNCH_CHECK();
  BiasJobs jobs{};
  jobs.n = L;
  // output layer: dW^T [in][16] = H^T dY (M = width), stored transposed as dW
  {
    const auto &Ly = h->lay[L - 1];
    Epi e;
    e.n_store = kOutPad;
    e.m_rows = Ly.in;
    e.out_ft = h->g + Ly.w_off;
    e.ld_ft = Ly.in_k;
    rc = launch_gemm(h->st, h->Ht[L - 2], 0, 0, h->dYt, 0, 0, Ly.in, kOutPad, cap, e, h->err, h->wait_ns);
    if (rc) return rc;
    jobs.j[L - 1] = BiasJob{h->dYt.p, cap, h->g + Ly.b_off, kOutPad};
    // dH = dY W, then dZ = dH (1 - H^2) of the last hidden layer
    Epi d;
    d.dact = h->H[L - 2].p;
    d.ld_dact = h->H[L - 2].cols;
    d.n_store = Ly.in;
    d.m_rows = cap;
    d.out_b = h->dZ[L - 2].p;
    d.ld_b = h->dZ[L - 2].cols;
    d.out_bt = h->dZt[L - 2].p;
    d.ld_bt = h->dZt[L - 2].cols;
    rc = launch_gemm(h->st, h->dY, 0, 0, Ly.wtb, 0, 0, cap, Ly.in, kOutPad, d, h->err, h->wait_ns);
    if (rc) return rc;
  }
  for (int l = L - 2; l >= 0; --l) {
    const auto &Ly = h->lay[l];
    // dW [out][in_k] = dZ^T X_in: A = dZ^T [out][cap], B = X_in^T [in_k][cap]
    Epi e;
    e.n_store = Ly.in_k;
    e.m_rows = Ly.out;
    e.out_f = h->g + Ly.w_off;
    e.ld_f = Ly.in_k;
    const Mat &Bm = (l == 0) ? Xt : h->Ht[l - 1];
    rc = launch_gemm(h->st, h->dZt[l], 0, 0, Bm, 0, l == 0 ? row0 : 0, Ly.out, Ly.in_k, cap, e, h->err, h->wait_ns);
    if (rc) return rc;
    jobs.j[l] = BiasJob{h->dZt[l].p, cap, h->g + Ly.b_off, Ly.out};
    if (l > 0) {
      Epi d;
      d.dact = h->H[l - 1].p;
      d.ld_dact = h->H[l - 1].cols;
      d.n_store = Ly.in;
      d.m_rows = cap;
      d.out_b = h->dZ[l - 1].p;
      d.ld_b = h->dZ[l - 1].cols;
      d.out_bt = h->dZt[l - 1].p;
      d.ld_bt = h->dZt[l - 1].cols;
      rc = launch_gemm(h->st, h->dZ[l], 0, 0, Ly.wtb, 0, 0, cap, Ly.in, Ly.out, d, h->err, h->wait_ns);
      if (rc) return rc;
    }
  }
  dim3 grid(ceil_div((int64_t)std::max(h->p.width, kOutPad) * 32, 256), L);
  k_bias_grad<<<grid, 256, 0, h->st>>>(jobs, cap);
  OTF_LAUNCH_CHECK();
  return MD_OK;
}

int adam_step(mlp_handle *h) {
  h->t += 1;
  const double c1 = 1.0 - std::pow((double)h->p.beta1, (double)h->t);
  const double c2 = 1.0 - std::pow((double)h->p.beta2, (double)h->t);
  k_adam<<<ceil_div(h->np_pad, 256), 256, 0, h->st>>>(h->w, h->g, h->m1, h->m2, h->np_pad, h->table, h->p.lr,
                                                       h->p.beta1, h->p.beta2, h->p.eps, h->p.weight_decay,
                                                       (float)c1, (float)c2);
  OTF_LAUNCH_CHECK();
  return MD_OK;
}

// Copies caller rows (host or device) into a device buffer of `count` floats.
int to_device(mlp_handle *h, const float *src, int64_t count, int32_t mem, float **dst_owned, const float **dst) {
  if (mem == MD_MEM_DEVICE) {
    *dst = src;
    *dst_owned = nullptr;
    return MD_OK;
  }
  if (mem != MD_MEM_HOST) {
    set_error("mem must be MD_MEM_HOST or MD_MEM_DEVICE");
    return MD_EINVAL;
  }
  OTF_CUDA(cudaMalloc(dst_owned, sizeof(float) * std::max<int64_t>(count, 1)));
  OTF_CUDA(cudaMemcpyAsync(*dst_owned, src, sizeof(float) * count, cudaMemcpyHostToDevice, h->st));
  *dst = *dst_owned;
  return MD_OK;
}

int grow_inference(mlp_handle *h, int64_t rows) {
  const int64_t need = ((rows + kBM - 1) / kBM) * kBM;
  if (need <= h->icap) return MD_OK;
  mat_free(h->xi);
  mat_free(h->hi[0]);
  mat_free(h->hi[1]);
  if (h->Yi) cudaFree(h->Yi);
  h->Yi = nullptr;
  h->icap = 0;
  int rc = mat_alloc(h->xi, need, h->k_in, kBM);
  if (!rc) rc = mat_alloc(h->hi[0], need, h->p.width, kBM);
  if (!rc) rc = mat_alloc(h->hi[1], need, h->p.width, kBM);
  if (rc) return rc;
  OTF_CUDA(cudaMalloc(&h->Yi, sizeof(float) * need * kOutPad));
  h->icap = need;
  return MD_OK;
}

void destroy(mlp_handle *h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  for (auto &Ly : h->lay) {
    mat_free(Ly.wb);
    mat_free(Ly.wtb);
  }
  for (auto *v : {&h->H, &h->Ht, &h->dZ, &h->dZt})
    for (auto &M : *v) mat_free(M);
  mat_free(h->xb);
  mat_free(h->xbt);
  mat_free(h->dY);
  mat_free(h->dYt);
  mat_free(h->xi);
  mat_free(h->hi[0]);
  mat_free(h->hi[1]);
  for (void *q : {(void *)h->w, (void *)h->g, (void *)h->m1, (void *)h->m2, (void *)h->xmean, (void *)h->xstd,
                  (void *)h->ymean, (void *)h->ystd, (void *)h->Y, (void *)h->T, (void *)h->loss, (void *)h->err,
                  (void *)h->Yi})
    if (q) cudaFree(q);
  if (h->err_host) cudaFreeHost(h->err_host);
  delete h;
}

// Shared-memory plan of the fused forward: layer l's weight panels (64
// columns x out_p rows each) back to back, then two activation tiles, then
// the bias and scaler tables and the barriers.
int setup_fused(mlp_handle *h) {
  FusedArgs &a = h->fa;
  a.L = h->L;
  a.n_in = h->p.n_in;
  a.k_in = h->k_in;
  a.n_out = h->p.n_out;
  uint32_t off = 0;
  int boff = 0, maxp = 2;
  for (int l = 0; l < h->L; ++l) {
    const auto &Ly = h->lay[l];
    const int np = (Ly.in_k + kBK - 1) / kBK;
    a.in_k[l] = Ly.in_k;
    a.out_p[l] = Ly.out_p;
    a.w_off[l] = off;
    off += (uint32_t)np * (uint32_t)Ly.out_p * 128u;
    a.b_off[l] = boff;
    boff += Ly.out_p;
    a.bias[l] = h->w + Ly.b_off;
    h->fm.w[l] = Ly.wb.map;
    maxp = std::max(maxp, np);
  }
  a.w_bytes = off;
  a.act_bytes = (uint32_t)maxp * kPanelBytes;
  a.nbias = boff;
  a.xmean = h->xmean;
  a.xstd = h->xstd;
  a.ymean = h->ymean;
  a.ystd = h->ystd;
  const size_t need = 1024 + (size_t)off + 2 * (size_t)a.act_bytes + fused_tables_bytes(boff, a.k_in) + 128;
  int dev = 0, optin = 0;
  OTF_CUDA(cudaGetDevice(&dev));
  OTF_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  OTF_CUDA(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev));
  h->fused = h->p.width == kBM && need <= (size_t)optin;
  h->fused_smem = need;
  if (h->fused) OTF_CUDA(cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  return MD_OK;
}

int create_impl(mlp_handle *h) {
  const mlp_params &p = h->p;
  h->L = p.depth + 1;
  h->k_in = std::max(64, (p.n_in + 15) / 16 * 16);
  h->cap = p.batch;
  h->lay.resize(h->L);
  int64_t off = 0, flat = 0;
  for (int l = 0; l < h->L; ++l) {
    auto &Ly = h->lay[l];
    Ly.in = l == 0 ? p.n_in : p.width;
    Ly.in_k = l == 0 ? h->k_in : p.width;
    Ly.out = l == h->L - 1 ? p.n_out : p.width;
    Ly.out_p = l == h->L - 1 ? kOutPad : p.width;
    Ly.w_off = off;
    off += (int64_t)Ly.out_p * Ly.in_k;
    Ly.b_off = off;
    off += Ly.out_p;
    flat += (int64_t)Ly.out * Ly.in + Ly.out;
    int rc = mat_alloc(Ly.wb, Ly.out_p, Ly.in_k, (uint32_t)Ly.out_p);
    if (rc) return rc;
    if (l > 0) {  // W^T feeds dH = dZ W; the output layer's is padded to 64 columns
      rc = mat_alloc(Ly.wtb, Ly.in_k, l == h->L - 1 ? 64 : Ly.out_p, (uint32_t)Ly.in_k);
      if (rc) return rc;
    }
    h->table.l[l] = AdamLayer{Ly.w_off, Ly.b_off, Ly.out_p, Ly.in_k, Ly.wb.p, Ly.wtb.p, (int)Ly.wtb.cols};
  }
  h->table.n = h->L;
  h->np_pad = off;
  h->np_flat = flat;
  for (float **q : {&h->w, &h->g, &h->m1, &h->m2}) {
    OTF_CUDA(cudaMalloc(q, sizeof(float) * off));
    OTF_CUDA(cudaMemset(*q, 0, sizeof(float) * off));
  }
  OTF_CUDA(cudaMalloc(&h->xmean, sizeof(float) * p.n_in));
  OTF_CUDA(cudaMalloc(&h->xstd, sizeof(float) * p.n_in));
  OTF_CUDA(cudaMalloc(&h->ymean, sizeof(float) * kOutPad));
  OTF_CUDA(cudaMalloc(&h->ystd, sizeof(float) * kOutPad));
  h->h_xmean.assign(p.n_in, 0.f);
  h->h_xstd.assign(p.n_in, 1.f);
  h->h_ymean.assign(p.n_out, 0.f);
  h->h_ystd.assign(p.n_out, 1.f);
  int rc = upload_scaler(h);
  if (rc) return rc;
  // Glorot-uniform weights from SplitMix64: layer l draws stream seed*1000 + 2l
  std::vector<float> flatv((size_t)flat);
  int64_t f = 0;
  for (int l = 0; l < h->L; ++l) {
    const auto &Ly = h->lay[l];
    const double lim = std::sqrt(6.0 / (Ly.in + Ly.out));
    const uint64_t s = p.seed * 1000ull + 2ull * l;
    for (int64_t k = 0; k < (int64_t)Ly.out * Ly.in; ++k)
      flatv[(size_t)f++] = (float)((2.0 * uniform01_at(s, (uint64_t)k + 1) - 1.0) * lim);
    for (int o = 0; o < Ly.out; ++o) flatv[(size_t)f++] = 0.f;
  }
  std::vector<float> pad;
  flat_to_pad(h, flatv.data(), pad);
  OTF_CUDA(cudaMemcpyAsync(h->w, pad.data(), sizeof(float) * off, cudaMemcpyHostToDevice, h->st));
  OTF_CUDA(cudaStreamSynchronize(h->st));
  rc = cast_weights(h);
  if (rc) return rc;
  // training batch buffers
  const int cap = h->cap, nh = p.depth;
  rc = mat_alloc(h->xb, cap, h->k_in, kBM);
  if (!rc) rc = mat_alloc(h->xbt, h->k_in, cap, (uint32_t)h->k_in);
  if (rc) return rc;
  h->H.resize(nh);
  h->Ht.resize(nh);
  h->dZ.resize(nh);
  h->dZt.resize(nh);
  for (int l = 0; l < nh; ++l) {
    rc = mat_alloc(h->H[l], cap, p.width, kBM);
    if (!rc) rc = mat_alloc(h->Ht[l], p.width, cap, (uint32_t)p.width);  // A of dW_out (box 128) / B of dW
    if (!rc) rc = mat_alloc(h->dZ[l], cap, p.width, kBM);
    if (!rc) rc = mat_alloc(h->dZt[l], p.width, cap, kBM);
    if (rc) return rc;
  }
  rc = mat_alloc(h->dY, cap, 64, kBM);
  if (!rc) rc = mat_alloc(h->dYt, kOutPad, cap, kOutPad);
  if (rc) return rc;
  OTF_CUDA(cudaMalloc(&h->Y, sizeof(float) * cap * kOutPad));
  OTF_CUDA(cudaMalloc(&h->T, sizeof(float) * cap * p.n_out));
  OTF_CUDA(cudaMalloc(&h->loss, sizeof(double) * 2));
  OTF_CUDA(cudaMemset(h->loss, 0, sizeof(double) * 2));
  OTF_CUDA(cudaMalloc(&h->err, sizeof(unsigned)));
  OTF_CUDA(cudaMemset(h->err, 0, sizeof(unsigned)));
  OTF_CUDA(cudaMallocHost(&h->err_host, sizeof(unsigned)));
  *h->err_host = 0u;
  OTF_CUDA(cudaDeviceSynchronize());
  return setup_fused(h);
}

// One launch over all rows: inputs read once, outputs written once.
int forward_fused(mlp_handle *h, const float *X, int64_t rows, float *Y, int32_t mem) {
  float *own = nullptr, *own_y = nullptr;
  const float *dX = nullptr;
  int rc = to_device(h, X, rows * h->p.n_in, mem, &own, &dX);
  float *dY = Y;
  if (!rc && mem == MD_MEM_HOST) {
    if (cudaMalloc(&own_y, sizeof(float) * rows * h->p.n_out) != cudaSuccess) {
      set_error("mlp_forward: output buffer allocation failed");
      rc = MD_ENOMEM;
    }
    dY = own_y;
  }
  if (!rc) {
    const int64_t tiles = (rows + kBM - 1) / kBM;
    const int grid = (int)std::min<int64_t>((tiles + 1) / 2, std::max(h->nsm, 1));
    FusedArgs a = h->fa;
    a.unscale = 1;
    k_mlp_fused<<<grid, kFusedThreads, h->fused_smem, h->st>>>(h->fm, a, dX, rows, dY, h->err);
    if (cudaGetLastError() != cudaSuccess) {
      set_error("k_mlp_fused launch failed");
      rc = MD_ECUDA;
    }
  }
  if (!rc && mem == MD_MEM_HOST &&
      cudaMemcpyAsync(Y, own_y, sizeof(float) * rows * h->p.n_out, cudaMemcpyDeviceToHost, h->st) != cudaSuccess) {
    set_error("mlp_forward: output copy failed");
    rc = MD_ECUDA;
  }
  if (!rc) rc = check_err(h);
  cudaStreamSynchronize(h->st);
  if (own) cudaFree(own);
  if (own_y) cudaFree(own_y);
  return rc;
}

}  // namespace

extern "C" {

int mlp_create(const mlp_params *p, void *cuda_stream, mlp_handle **out) {
  clear_error();
  if (!p || !out) {
    set_error("mlp_create: null argument");
    return MD_EINVAL;
  }
  *out = nullptr;
  if (p->n_in < 1 || p->n_in > 240 || p->width != 128 || p->depth < 1 || p->depth > kMaxLayers - 2 ||
      p->n_out < 1 || p->n_out > kOutPad || p->batch < kBM || p->batch % kBM || p->batch > 4096) {
    set_error("mlp_create: need 1 <= n_in <= 240, width = 128, 1 <= depth <= 6, 1 <= n_out <= 16 and a batch "
              "that is a multiple of 128 up to 4096");
    return MD_EINVAL;
  }
  if (!(p->lr > 0) || !(p->beta1 >= 0 && p->beta1 < 1) || !(p->beta2 >= 0 && p->beta2 < 1) || !(p->eps > 0) ||
      !(p->weight_decay >= 0)) {
    set_error("mlp_create: Adam needs lr > 0, 0 <= beta < 1, eps > 0, weight_decay >= 0");
    return MD_EINVAL;
  }
  mlp_handle *h = new (std::nothrow) mlp_handle_s;
  if (!h) return MD_ENOMEM;
  h->p = *p;
  h->st = (cudaStream_t)cuda_stream;
  int rc = create_impl(h);
  if (rc) {
    destroy(h);
    return rc;
  }
  *out = h;
  return MD_OK;
}

int mlp_param_count(const mlp_handle *h, int64_t *count) {
  if (!h || !count) return MD_EINVAL;
  *count = h->np_flat;
  return MD_OK;
}

int mlp_get_params(mlp_handle *h, float *flat, int64_t count, int32_t mem) {
  clear_error();
  if (!h || !flat || count != h->np_flat) {
    set_error("mlp_get_params: null argument or count != %lld", h ? (long long)h->np_flat : 0LL);
    return MD_EINVAL;
  }
  std::vector<float> pad((size_t)h->np_pad), f((size_t)count);
  OTF_CUDA(cudaMemcpyAsync(pad.data(), h->w, sizeof(float) * h->np_pad, cudaMemcpyDeviceToHost, h->st));
  OTF_CUDA(cudaStreamSynchronize(h->st));
  pad_to_flat(h, pad, f.data());
  if (mem == MD_MEM_HOST) {
    std::memcpy(flat, f.data(), sizeof(float) * count);
  } else {
    OTF_CUDA(cudaMemcpyAsync(flat, f.data(), sizeof(float) * count, cudaMemcpyHostToDevice, h->st));
    OTF_CUDA(cudaStreamSynchronize(h->st));
  }
  return MD_OK;
}

int mlp_set_params(mlp_handle *h, const float *flat, int64_t count, int32_t mem) {
  clear_error();
  if (!h || !flat || count != h->np_flat) {
    set_error("mlp_set_params: null argument or count != %lld", h ? (long long)h->np_flat : 0LL);
    return MD_EINVAL;
  }
  std::vector<float> f((size_t)count), pad;
  if (mem == MD_MEM_HOST) {
    std::memcpy(f.data(), flat, sizeof(float) * count);
  } else {
    OTF_CUDA(cudaMemcpyAsync(f.data(), flat, sizeof(float) * count, cudaMemcpyDeviceToHost, h->st));
    OTF_CUDA(cudaStreamSynchronize(h->st));
  }
  flat_to_pad(h, f.data(), pad);
  OTF_CUDA(cudaMemcpyAsync(h->w, pad.data(), sizeof(float) * h->np_pad, cudaMemcpyHostToDevice, h->st));
  OTF_CUDA(cudaStreamSynchronize(h->st));
  int rc = reset_adam(h);
  if (!rc) rc = cast_weights(h);
  if (!rc) {
    OTF_CUDA(cudaStreamSynchronize(h->st));
  }
  return rc;
}

int mlp_set_scaler(mlp_handle *h, const float *x_mean, const float *x_std, const float *y_mean, const float *y_std) {
  clear_error();
  if (!h || !x_mean || !x_std || !y_mean || !y_std) {
    set_error("mlp_set_scaler: null argument");
    return MD_EINVAL;
  }
  for (int i = 0; i < h->p.n_in; ++i)
    if (!(x_std[i] > 0)) {
      set_error("mlp_set_scaler: x_std[%d] is not positive", i);
      return MD_EINVAL;
    }
  for (int i = 0; i < h->p.n_out; ++i)
    if (!(y_std[i] > 0)) {
      set_error("mlp_set_scaler: y_std[%d] is not positive", i);
      return MD_EINVAL;
    }
  h->h_xmean.assign(x_mean, x_mean + h->p.n_in);
  h->h_xstd.assign(x_std, x_std + h->p.n_in);
  h->h_ymean.assign(y_mean, y_mean + h->p.n_out);
  h->h_ystd.assign(y_std, y_std + h->p.n_out);
  return upload_scaler(h);
}

int mlp_fit_scaler(mlp_handle *h, const float *X, const float *T, int64_t rows) {
  clear_error();
  if (!h || !X || !T || rows < 1) {
    set_error("mlp_fit_scaler: null argument or rows < 1");
    return MD_EINVAL;
  }
  auto stats = [&](const float *A, int cols, std::vector<float> &mean, std::vector<float> &sd) {
    mean.assign(cols, 0.f);
    sd.assign(cols, 1.f);
    for (int c = 0; c < cols; ++c) {
      double s = 0.0, s2 = 0.0;
      for (int64_t r = 0; r < rows; ++r) s += A[r * cols + c];
      const double mu = s / rows;
      for (int64_t r = 0; r < rows; ++r) {
        const double d = A[r * cols + c] - mu;
        s2 += d * d;
      }
      const double v = std::sqrt(s2 / rows);
      mean[c] = (float)mu;
      sd[c] = v > 0 ? (float)v : 1.f;
    }
  };
  stats(X, h->p.n_in, h->h_xmean, h->h_xstd);
  stats(T, h->p.n_out, h->h_ymean, h->h_ystd);
  return upload_scaler(h);
}

int mlp_forward(mlp_handle *h, const float *X, int64_t rows, float *Y, int32_t mem) {
  clear_error();
  if (!h || !X || !Y || rows < 1) {
    set_error("mlp_forward: null argument or rows < 1");
    return MD_EINVAL;
  }
  if (h->fused) return forward_fused(h, X, rows, Y, mem);
  const int64_t chunk = 65536;  // rows per pass (about 60 MB of bfloat16 activations)
  int rc = grow_inference(h, std::min(rows, chunk));
  if (rc) return rc;
  float *own = nullptr;
  const float *dX = nullptr;
  rc = to_device(h, X, rows * h->p.n_in, mem, &own, &dX);
  if (rc) return rc;
  for (int64_t r0 = 0; r0 < rows && !rc; r0 += chunk) {
    const int64_t n = std::min(chunk, rows - r0);
    const int64_t npad = (n + kBM - 1) / kBM * kBM;
    k_prep_x<<<std::min<int64_t>(1024, ceil_div(npad * h->k_in, 256)), 256, 0, h->st>>>(
        dX + r0 * h->p.n_in, n, h->p.n_in, h->xmean, h->xstd, h->xi.p, npad, h->k_in, nullptr, 0);
    if (cudaGetLastError() != cudaSuccess) {
      rc = MD_ECUDA;
      set_error("k_prep_x launch failed");
      break;
    }
    rc = forward(h, h->xi, 0, n, h->hi, 2, nullptr, h->Yi, true);
    if (rc) break;
    const cudaMemcpyKind kind = mem == MD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (cudaMemcpy2DAsync(Y + r0 * h->p.n_out, sizeof(float) * h->p.n_out, h->Yi, sizeof(float) * kOutPad,
                          sizeof(float) * h->p.n_out, n, kind, h->st) != cudaSuccess) {
      rc = MD_ECUDA;
      set_error("mlp_forward: output copy failed");
    }
  }
  if (!rc) rc = check_err(h);
  cudaStreamSynchronize(h->st);
  if (own) cudaFree(own);
  return rc;
}

int mlp_loss_grad(mlp_handle *h, const float *X, const float *T, int64_t rows, double *loss, float *grad,
                  int32_t mem) {
  clear_error();
  if (!h || !X || !T || rows != h->cap) {
    set_error("mlp_loss_grad: null argument or rows != batch (%d)", h ? h->cap : 0);
    return MD_EINVAL;
  }
  float *ox = nullptr, *ot = nullptr;
  const float *dX = nullptr, *dT = nullptr;
  int rc = to_device(h, X, rows * h->p.n_in, mem, &ox, &dX);
  if (!rc) rc = to_device(h, T, rows * h->p.n_out, mem, &ot, &dT);
  if (!rc) {
    k_prep_x<<<std::min<int64_t>(1024, ceil_div(rows * h->k_in, 256)), 256, 0, h->st>>>(
        dX, rows, h->p.n_in, h->xmean, h->xstd, h->xb.p, rows, h->k_in, h->xbt.p, h->xbt.cols);
    k_prep_t<<<ceil_div(rows * h->p.n_out, 256), 256, 0, h->st>>>(dT, rows, h->p.n_out, h->ymean, h->ystd, h->T);
    if (cudaGetLastError() != cudaSuccess) {
      set_error("input preparation launch failed");
      rc = MD_ECUDA;
    }
  }
  if (!rc) rc = train_step(h, h->xb, h->xbt, 0, h->T, 0.0);
  double lv[2] = {0, 0};
  if (!rc && cudaMemcpyAsync(lv, h->loss, sizeof(lv), cudaMemcpyDeviceToHost, h->st) != cudaSuccess) rc = MD_ECUDA;
  if (!rc) rc = check_err(h);
  if (!rc && loss) *loss = lv[1];
  if (!rc && grad) {
    std::vector<float> pad((size_t)h->np_pad), f((size_t)h->np_flat);
    if (cudaMemcpyAsync(pad.data(), h->g, sizeof(float) * h->np_pad, cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
        cudaStreamSynchronize(h->st) != cudaSuccess) {
      rc = MD_ECUDA;
    } else {
      pad_to_flat(h, pad, f.data());
      if (mem == MD_MEM_HOST)
        std::memcpy(grad, f.data(), sizeof(float) * h->np_flat);
      else if (cudaMemcpy(grad, f.data(), sizeof(float) * h->np_flat, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = MD_ECUDA;
    }
  }
  cudaStreamSynchronize(h->st);
  if (ox) cudaFree(ox);
  if (ot) cudaFree(ot);
  if (rc == MD_ECUDA && !md_last_error()[0]) set_error("mlp_loss_grad: CUDA call failed");
  return rc;
}

int mlp_adam_step(mlp_handle *h, const float *grad, int32_t mem) {
  clear_error();
  if (!h) return MD_EINVAL;
  if (grad) {
    std::vector<float> f((size_t)h->np_flat), pad;
    if (mem == MD_MEM_HOST) {
      std::memcpy(f.data(), grad, sizeof(float) * h->np_flat);
    } else {
      OTF_CUDA(cudaMemcpyAsync(f.data(), grad, sizeof(float) * h->np_flat, cudaMemcpyDeviceToHost, h->st));
      OTF_CUDA(cudaStreamSynchronize(h->st));
    }
    flat_to_pad(h, f.data(), pad);
    OTF_CUDA(cudaMemcpyAsync(h->g, pad.data(), sizeof(float) * h->np_pad, cudaMemcpyHostToDevice, h->st));
  }
  int rc = adam_step(h);
  if (!rc) {
    OTF_CUDA(cudaStreamSynchronize(h->st));
  }
  return rc;
}

int mlp_train(mlp_handle *h, const float *X, const float *T, int64_t rows, int32_t epochs, const int64_t *order,
              uint64_t shuffle_seed, double *loss_per_epoch, int32_t mem) {
  clear_error();
  if (!h || !X || !T || epochs < 0) {
    set_error("mlp_train: null argument or epochs < 0");
    return MD_EINVAL;
  }
  const int cap = h->cap;
  const int64_t nb = rows / cap;  // batches per epoch
  if (nb < 1) {
    set_error("mlp_train: %lld rows hold no full batch of %d", (long long)rows, cap);
    return MD_EINVAL;
  }
  if (rows > ((int64_t)1 << 30) / h->k_in) {
    set_error("mlp_train: too many rows");
    return MD_EINVAL;
  }
  const int64_t nused = nb * cap;
  Mat Xall, Xs, Xst;
  float *Tall = nullptr, *Ts = nullptr, *ox = nullptr, *ot = nullptr;
  int64_t *dperm = nullptr;
  double *dloss = nullptr;
  const float *dX = nullptr, *dT = nullptr;
  std::vector<double> hist((size_t)epochs, 0.0);
  int rc = to_device(h, X, rows * h->p.n_in, mem, &ox, &dX);
  if (!rc) rc = to_device(h, T, rows * h->p.n_out, mem, &ot, &dT);
  if (!rc) rc = mat_alloc(Xall, rows, h->k_in, kBM);
  if (!rc) rc = mat_alloc(Xs, nused, h->k_in, kBM);
  if (!rc) rc = mat_alloc(Xst, h->k_in, nused, (uint32_t)h->k_in);
  auto cuda_ok = [&](cudaError_t e) {
    if (e != cudaSuccess && !rc) {
      set_error("mlp_train: %s", cudaGetErrorString(e));
      rc = e == cudaErrorMemoryAllocation ? MD_ENOMEM : MD_ECUDA;
    }
    return rc == MD_OK;
  };
  if (!rc) cuda_ok(cudaMalloc(&Tall, sizeof(float) * rows * h->p.n_out));
  if (!rc) cuda_ok(cudaMalloc(&Ts, sizeof(float) * nused * h->p.n_out));
  if (!rc) cuda_ok(cudaMalloc(&dperm, sizeof(int64_t) * rows));
  if (!rc) cuda_ok(cudaMalloc(&dloss, sizeof(double) * std::max(epochs, 1)));
  if (!rc) cuda_ok(cudaMemsetAsync(dloss, 0, sizeof(double) * std::max(epochs, 1), h->st));
  if (!rc) {
    k_prep_x<<<1024, 256, 0, h->st>>>(dX, rows, h->p.n_in, h->xmean, h->xstd, Xall.p, rows, h->k_in, nullptr, 0);
    k_prep_t<<<256, 256, 0, h->st>>>(dT, rows, h->p.n_out, h->ymean, h->ystd, Tall);
    cuda_ok(cudaGetLastError());
  }
  if (!rc) cuda_ok(cudaMemsetAsync(h->loss, 0, sizeof(double), h->st));
  std::vector<int64_t> perm((size_t)rows);
  std::vector<uint64_t> keys((size_t)rows);
  for (int e = 0; e < epochs && !rc; ++e) {
    if (order) {
      std::memcpy(perm.data(), order + (int64_t)e * rows, sizeof(int64_t) * rows);
      for (int64_t i = 0; i < rows; ++i)
        if (perm[(size_t)i] < 0 || perm[(size_t)i] >= rows) {
          set_error("mlp_train: order[%d][%lld] out of range", e, (long long)i);
          rc = MD_EINVAL;
          break;
        }
      if (rc) break;
    } else {  // sort SplitMix64 keys of stream shuffle_seed + e (ties by index)
      for (int64_t i = 0; i < rows; ++i) {
        keys[(size_t)i] = splitmix64_at(shuffle_seed + (uint64_t)e, (uint64_t)i + 1);
        perm[(size_t)i] = i;
      }
      std::stable_sort(perm.begin(), perm.end(),
                       [&](int64_t a, int64_t b) { return keys[(size_t)a] < keys[(size_t)b]; });
    }
    if (!cuda_ok(cudaMemcpyAsync(dperm, perm.data(), sizeof(int64_t) * rows, cudaMemcpyHostToDevice, h->st))) break;
    k_gather<<<1024, 256, 0, h->st>>>(Xall.p, Tall, dperm, nused, h->k_in, h->p.n_out, Xs.p, Xst.p, Ts);
    if (!cuda_ok(cudaGetLastError())) break;
    for (int64_t b = 0; b < nb && !rc; ++b) {
      // the loss kernel adds loss / nb to the epoch's slot via h->loss[0]
      rc = train_step(h, Xs, Xst, (int)(b * cap), Ts + b * cap * h->p.n_out, 1.0 / (double)nb);
      if (!rc) rc = adam_step(h);
    }
    if (!rc) cuda_ok(cudaMemcpyAsync(dloss + e, h->loss, sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    if (!rc) cuda_ok(cudaMemsetAsync(h->loss, 0, sizeof(double), h->st));
    if (!rc) cuda_ok(cudaStreamSynchronize(h->st));  // the host permutation buffer is reused next epoch
  }
  if (!rc && epochs > 0)
    cuda_ok(cudaMemcpyAsync(hist.data(), dloss, sizeof(double) * epochs, cudaMemcpyDeviceToHost, h->st));
  if (!rc) rc = check_err(h);
  cudaStreamSynchronize(h->st);
  if (!rc && loss_per_epoch) std::memcpy(loss_per_epoch, hist.data(), sizeof(double) * epochs);
  mat_free(Xall);
  mat_free(Xs);
  mat_free(Xst);
  for (void *q : {(void *)Tall, (void *)Ts, (void *)ox, (void *)ot, (void *)dperm, (void *)dloss})
    if (q) cudaFree(q);
  return rc;
}

int mlp_set_wait_limit(mlp_handle *h, int64_t ns) {
  clear_error();
  if (!h || ns < 0) {
    set_error("mlp_set_wait_limit: null handle or negative limit");
    return MD_EINVAL;
  }
  h->wait_ns = (uint64_t)ns;
  return MD_OK;
}

void mlp_free(mlp_handle *h) { destroy(h); }

int gk_tail_features(const double *c_sigma, const double *c_q, int64_t ld, int64_t nruns, const double *volume,
                     const double *temperature, const double *density, float *out) {
  clear_error();
  constexpr int kPts = 64;
  if (!c_sigma || !c_q || !volume || !temperature || !density || !out || ld < kPts || nruns < 0) {
    set_error("gk_tail_features: null argument or fewer than 64 readout points");
    return MD_EINVAL;
  }
  for (int64_t r = 0; r < nruns; ++r) {
    const double *cs = c_sigma + r * ld, *cq = c_q + r * ld;
    const double V = volume[r], T = temperature[r];
    if (!(cs[0] > 0) || !(cq[0] > 0) || !(V > 0) || !(T > 0)) {
      set_error("gk_tail_features: run %lld has a non-positive C(0), volume or temperature", (long long)r);
      return MD_EINVAL;
    }
    float *o = out + r * (2 * kPts + 4);
    for (int i = 0; i < kPts; ++i) o[i] = (float)(cs[i] / cs[0]);
    o[kPts] = (float)std::log(V * cs[0] / T);
    for (int i = 0; i < kPts; ++i) o[kPts + 1 + i] = (float)(cq[i] / cq[0]);
    o[2 * kPts + 1] = (float)std::log(V * cq[0] / (T * T));
    o[2 * kPts + 2] = (float)T;
    o[2 * kPts + 3] = (float)density[r];
  }
  return MD_OK;
}

int gk_tail_box(const double *temperature, const double *density, int64_t n, gk_tail_rule *rule) {
  clear_error();
  if (!temperature || !density || !rule || n < 1) {
    set_error("gk_tail_box: null argument or no runs");
    return MD_EINVAL;
  }
  rule->T_min = rule->T_max = temperature[0];
  rule->rho_min = rule->rho_max = density[0];
  for (int64_t r = 1; r < n; ++r) {
    rule->T_min = std::min(rule->T_min, temperature[r]);
    rule->T_max = std::max(rule->T_max, temperature[r]);
    rule->rho_min = std::min(rule->rho_min, density[r]);
    rule->rho_max = std::max(rule->rho_max, density[r]);
  }
  return MD_OK;
}

int gk_tail_rms_rel(const double *a, const double *b, const double *w, int64_t n, double *out) {
  clear_error();
  if (!a || !b || !out || n < 1) {
    set_error("gk_tail_rms_rel: null argument or no values");
    return MD_EINVAL;
  }
  double s = 0.0;
  for (int64_t r = 0; r < n; ++r) {
    if (!(b[r] != 0.0)) {
      set_error("gk_tail_rms_rel: reference value %lld is zero", (long long)r);
      return MD_EINVAL;
    }
    const double e = (a[r] - b[r]) / b[r];
    s += e * e * (w ? w[r] : 1.0);
  }
  *out = std::sqrt(s / (double)n);
  return MD_OK;
}

int gk_tail_choose(const gk_tail_rule *rule, const double *temperature, const double *density, const double *steps,
                   const double *net, const double *own, int64_t nruns, double *out, int32_t *used) {
  clear_error();
  if (!rule || !temperature || !density || !steps || !net || !own || !out || nruns < 0) {
    set_error("gk_tail_choose: null argument");
    return MD_EINVAL;
  }
  for (int64_t r = 0; r < nruns; ++r) {
    if (!(steps[r] > 0.0)) {
      set_error("gk_tail_choose: run %lld has no correlated steps", (long long)r);
      return MD_EINVAL;
    }
    const bool inside = temperature[r] >= rule->T_min && temperature[r] <= rule->T_max &&
                        density[r] >= rule->rho_min && density[r] <= rule->rho_max;
    const double root = std::sqrt(steps[r]);
    for (int k = 0; k < 2; ++k) {
      const bool use = inside && rule->short_coeff[k] / root > rule->net_error[k];
      out[2 * r + k] = use ? net[2 * r + k] : own[2 * r + k];
      if (used) used[2 * r + k] = use ? 1 : 0;
    }
  }
  return MD_OK;
}

}  // extern "C"
