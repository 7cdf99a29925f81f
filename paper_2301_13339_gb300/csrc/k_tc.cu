// Tensor-core (tcgen05) building blocks for sm_103a, written as inline PTX:
// operands staged in shared memory in the canonical no-swizzle K-major
// layout (core matrices of 8 rows x 16 bytes), accumulators in tensor memory
// (TMEM), MMAs issued by one thread and tracked by an mbarrier, results read
// back with tcgen05.ld.
//
// Layout of a K-major operand tile (rows x 8 TF32 elements per MMA step):
// element (row, k) at byte (row % 8) * 16 + (row / 8) * SBO + (k / 4) * LBO +
// (k % 4) * 4, with LBO = 128 (the two 16-byte halves of a row's 32 bytes)
// and SBO = 256 (the next group of 8 rows).
//
// Every wait is bounded: after TC_SPIN_LIMIT polls the kernel records an
// error, still frees its TMEM and returns.
#include "qtt_internal.cuh"
#include <cstdint>

namespace qtt {

constexpr int TC_SPIN_LIMIT = 1 << 22;
constexpr uint32_t TC_LBO = 128, TC_SBO = 256;

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (all in 16-byte units), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::tf32: D in FP32, A and B TF32, both
// K-major, shape M x N
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tc_mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// wait for the phase of the mbarrier to complete; false after the spin limit
__device__ __forceinline__ bool tc_mbar_wait(uint32_t mbar, uint32_t phase) {
  for (int it = 0; it < TC_SPIN_LIMIT; ++it) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of element (row, k) (k < 8) inside one K-step operand tile
__device__ __forceinline__ uint32_t tc_tile_off(int row, int k) {
  return (uint32_t)((row & 7) * 16 + (row >> 3) * TC_SBO + (k >> 2) * TC_LBO + (k & 3) * 4);
}

// Self-test GEMM: C (128 x N, row-major) = A (128 x K, row-major) B^T with
// B (N x K, row-major); N in {32, 64, 128, 256}, K a multiple of 8.  One CTA
// of 128 threads (four warps: warp w reads TMEM lanes 32w..32w+31); one
// 8-deep K step per MMA.  *err receives 1 if a wait ran out.
__global__ void __launch_bounds__(128)
k_tc_selftest(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ C,
              int N, int K, int* err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  float* As = reinterpret_cast<float*>(tc_smem);                  // 128 x 8  (4 KB)
  float* Bs = reinterpret_cast<float*>(tc_smem + 128 * 8 * 4);    // N x 8    (<= 8 KB)
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t ncols = (uint32_t)N;   // power of two >= 32
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc_smem_u32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) tc_mbar_init(tc_smem_u32(&mbar), 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = tc_idesc_tf32(128, N);
  bool ok = true;
  uint32_t phase = 0;
  for (int k0 = 0; k0 < K && ok; k0 += 8) {
    // stage the K step: thread t writes row t of A and rows t, t+128 of B
    for (int k = 0; k < 8; ++k) {
      As[tc_tile_off(tid, k) / 4] = A[(size_t)tid * K + k0 + k];
      for (int r = tid; r < N; r += 128) Bs[tc_tile_off(r, k) / 4] = B[(size_t)r * K + k0 + k];
    }
    tc_fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      tc_mma_tf32(tmem, tc_sdesc(tc_smem_u32(As), TC_LBO, TC_SBO),
                  tc_sdesc(tc_smem_u32(Bs), TC_LBO, TC_SBO), idesc, k0 > 0 ? 1u : 0u);
      tc_commit(tc_smem_u32(&mbar));
    }
    ok = tc_mbar_wait(tc_smem_u32(&mbar), phase);
    phase ^= 1u;
    tc_fence_after();
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const int row = tid;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc_ld16(tmem + lane_base + (uint32_t)c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) C[(size_t)row * N + c0 + i] = v[i];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
}

}  // namespace qtt

using namespace qtt;

extern "C" qtt_status qtt_debug_tc_selftest(const float* A, const float* B, float* C, int N, int K,
                                            int* err_dev, void* stream) {
  clear_error();
  if (!A || !B || !C || !err_dev) {
    set_error("qtt_debug_tc_selftest: NULL argument");
    return QTT_EINVAL;
  }
  if (!(N == 32 || N == 64 || N == 128 || N == 256) || K < 8 || (K % 8) != 0) {
    set_error("qtt_debug_tc_selftest: N in {32, 64, 128, 256}, K a positive multiple of 8");
    return QTT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t sm = (size_t)(128 + 256) * 8 * 4;
  k_tc_selftest<<<1, 128, sm, s>>>(A, B, C, N, K, err_dev);
  return cuda_check(cudaGetLastError(), "qtt_debug_tc_selftest launch");
}
