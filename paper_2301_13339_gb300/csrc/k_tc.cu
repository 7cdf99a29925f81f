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

namespace qtt {

// ---------------------------------------------------------------------------
// Complex GEMM on the tensor cores, FP32-accurate: C = op(A) B with the
// strides and batching of CGemmArgs (A complex or real).
//
// The complex product is one real product over the stacking
//   A' rows 2i = [Re a_i, -Im a_i], 2i+1 = [Im a_i, Re a_i]   (real k 2k, 2k+1)
//   B' = [Re B; Im B] (in K-major rows: the interleaved complex storage)
// so that row 2i of C' = A' B' is Re C[i] and row 2i+1 Im C[i].  A CTA owns
// 64 complex rows (one M = 128 MMA) and TN_TC complex columns.  Each operand
// is split x ~ hi + lo, hi = x and lo = x - hi both rounded to nearest TF32,
// and hi hi + hi lo + lo hi are accumulated: products of 11-bit values are
// exact in FP32; the dropped lo lo term and the rounding of lo are near
// 2^-22 relative, without a sign bias.
//
// The tensor core's FP32 accumulator rounds one-signed, so it only sums one
// chunk of 8 complex k (two k-steps, 6 MMAs): every chunk accumulates into a
// fresh tensor-memory buffer, and the threads add the chunk sums into
// registers with Kahan compensation.  Two buffers alternate (shared memory
// and tensor memory): the MMAs of chunk c run while the threads read back
// chunk c - 1 and load chunk c + 1.  With split-K the partial of the tile
// goes to part (element (i, j) at i + M j) for a compensated sum.
constexpr int TN_TC = 64;              // complex columns per CTA (MMA N)
constexpr int TC_KC = 8;               // complex k per chunk
constexpr int TC_THREADS = 256;
constexpr int TC_A_TILE = 128 * 8 * 4;         // bytes of one A k-step tile (128 x 8 TF32)
constexpr int TC_B_TILE = TN_TC * 8 * 4;       // bytes of one B k-step tile
constexpr int TC_BUF = 4 * TC_A_TILE + 4 * TC_B_TILE;   // {hi, lo} x two k-steps
constexpr size_t TC_SMEM = 2 * (size_t)TC_BUF + 1024;
constexpr int TC_AE = 64 * TC_KC / TC_THREADS;      // A elements per thread and chunk (2)
constexpr int TC_BE = TN_TC * TC_KC / TC_THREADS;   // B elements per thread and chunk (2)
constexpr int TC_TCOLS = 2 * TN_TC;                  // tensor-memory columns (two buffers)
// longest k run of one CTA (single-batch products split k beyond it and add
// the partials with compensation; within a run the chunk sums are added
// with compensation too)
constexpr int TC_KMAX = 1024;

// x rounded to the nearest TF32 value (ties away from zero): the result
// has 11 significant bits, so the tensor core consumes it exactly
__device__ __forceinline__ float tc_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ float2 tc_load_a(const float* p, int) { return make_float2(__ldg(p), 0.f); }
__device__ __forceinline__ float2 tc_load_a(const float2* p, int conj) {
  const float2 v = __ldg(p);
  return make_float2(v.x, conj ? -v.y : v.y);
}

// hi and lo parts of v at (row, real k) of the chunk's {hi, lo} x step
// tiles: hi = tf32(v), lo = tf32(v - hi) (v - hi is exact in FP32), so both
// are exact TF32 operands and v - hi - lo is below 2^-22 |v|, unbiased
__device__ __forceinline__ void tc_put(unsigned char* tiles, int tile_bytes, int row, int kr, float v) {
  const int step = kr >> 3;
  const uint32_t off = tc_tile_off(row, kr & 7);
  const float hi = tc_tf32(v);
  *reinterpret_cast<float*>(tiles + (size_t)step * tile_bytes + off) = hi;
  *reinterpret_cast<float*>(tiles + (size_t)(2 + step) * tile_bytes + off) = tc_tf32(v - hi);
}

template <typename TA>
__global__ void __launch_bounds__(TC_THREADS, 2)
k_tc_cgemm(CGemmArgs<TA> g, int nbatch, int kchunk, float2* __restrict__ part, long long ldpart,
           int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char tc_dyn[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int bz = blockIdx.z % nbatch, split = blockIdx.z / nbatch;
  const int b1 = bz % g.nb1, b2 = bz / g.nb1;
  const TA* A = g.A + g.bA1 * b1 + g.bA2 * b2;
  const float2* B = g.B + g.bB1 * b1 + g.bB2 * b2;
  const long long i0 = (long long)blockIdx.y * 64, j0 = (long long)blockIdx.x * TN_TC;
  const int kbeg = split * kchunk;
  const int kend = min(g.K, kbeg + kchunk);
  const int nch = (kend > kbeg) ? (kend - kbeg + TC_KC - 1) / TC_KC : 0;
  unsigned char* base = tc_dyn + ((1024u - (tc_smem_u32(tc_dyn) & 1023u)) & 1023u);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc_smem_u32(&tmem_slot)),
                 "r"((uint32_t)TC_TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    tc_mbar_init(tc_smem_u32(&mbar[0]), 1);
    tc_mbar_init(tc_smem_u32(&mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = tc_idesc_tf32(128, TN_TC);
  // tensor-memory lanes of this warp, and its half of the columns
  const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
  const int half = warp >> 2;

  // this thread's elements of a chunk: A (ii, kk) and B (kk, jj)
  int a_ii[TC_AE], a_kk[TC_AE], b_kk[TC_BE], b_jj[TC_BE];
#pragma unroll
  for (int t = 0; t < TC_AE; ++t) {
    const int e = tid + t * TC_THREADS;
    if (g.sAi == 1) { a_ii[t] = e % 64; a_kk[t] = e / 64; }
    else { a_kk[t] = e % TC_KC; a_ii[t] = e / TC_KC; }
  }
#pragma unroll
  for (int t = 0; t < TC_BE; ++t) {
    const int e = tid + t * TC_THREADS;
    b_kk[t] = e % TC_KC;
    b_jj[t] = e / TC_KC;
  }
  float2 ra[TC_AE], rb[TC_BE];
  auto load_chunk = [&](int c) {
    const int k0 = kbeg + c * TC_KC;
#pragma unroll
    for (int t = 0; t < TC_AE; ++t) {
      const long long i = i0 + a_ii[t];
      const int k = k0 + a_kk[t];
      ra[t] = (i < g.M && k < kend) ? tc_load_a(A + i * g.sAi + (long long)k * g.sAk, g.conjA)
                                    : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < TC_BE; ++t) {
      const long long j = j0 + b_jj[t];
      const int k = k0 + b_kk[t];
      rb[t] = (j < g.N && k < kend) ? __ldg(B + (long long)k * g.sBk + j * g.sBj)
                                    : make_float2(0.f, 0.f);
    }
  };
  // compensated running sums of this thread's 32 outputs
  float sum[32], cmp[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) { sum[q] = 0.f; cmp[q] = 0.f; }
  auto flush = [&](int buf) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v[16];
      tc_ld16(tmem + lane_addr + (uint32_t)(TN_TC * buf + 32 * half + 16 * h), v);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float y = v[q] - cmp[16 * h + q];
        const float t = sum[16 * h + q] + y;
        cmp[16 * h + q] = (t - sum[16 * h + q]) - y;
        sum[16 * h + q] = t;
      }
    }
  };

  uint32_t phase[2] = {0u, 0u};
  bool ok = true;
  if (nch > 0) load_chunk(0);
  for (int c = 0; c < nch; ++c) {
    const int buf = c & 1;
    unsigned char* sa = base + (size_t)buf * TC_BUF;
    unsigned char* sb = sa + 4 * TC_A_TILE;
    // buffer buf was last used by chunk c - 2, whose MMAs completed (and
    // whose sums were read) in the previous iteration
#pragma unroll
    for (int t = 0; t < TC_AE; ++t) {
      const float2 a = ra[t];
      const int ii = a_ii[t], kr = 2 * a_kk[t];
      tc_put(sa, TC_A_TILE, 2 * ii, kr, a.x);
      tc_put(sa, TC_A_TILE, 2 * ii, kr + 1, -a.y);
      tc_put(sa, TC_A_TILE, 2 * ii + 1, kr, a.y);
      tc_put(sa, TC_A_TILE, 2 * ii + 1, kr + 1, a.x);
    }
#pragma unroll
    for (int t = 0; t < TC_BE; ++t) {
      tc_put(sb, TC_B_TILE, b_jj[t], 2 * b_kk[t], rb[t].x);
      tc_put(sb, TC_B_TILE, b_jj[t], 2 * b_kk[t] + 1, rb[t].y);
    }
    tc_fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t dacc = tmem + (uint32_t)(TN_TC * buf);
#pragma unroll
      for (int step = 0; step < 2; ++step) {
        const uint64_t dah = tc_sdesc(tc_smem_u32(sa + (size_t)step * TC_A_TILE), TC_LBO, TC_SBO);
        const uint64_t dal = tc_sdesc(tc_smem_u32(sa + (size_t)(2 + step) * TC_A_TILE), TC_LBO, TC_SBO);
        const uint64_t dbh = tc_sdesc(tc_smem_u32(sb + (size_t)step * TC_B_TILE), TC_LBO, TC_SBO);
        const uint64_t dbl = tc_sdesc(tc_smem_u32(sb + (size_t)(2 + step) * TC_B_TILE), TC_LBO, TC_SBO);
        tc_mma_tf32(dacc, dah, dbh, idesc, step > 0 ? 1u : 0u);   // a fresh sum per chunk
        tc_mma_tf32(dacc, dah, dbl, idesc, 1u);
        tc_mma_tf32(dacc, dal, dbh, idesc, 1u);
      }
      tc_commit(tc_smem_u32(&mbar[buf]));
    }
    if (c + 1 < nch) load_chunk(c + 1);
    if (c >= 1) {   // chunk c - 1: wait for its MMAs, add its sums
      const int pb = buf ^ 1;
      ok = __syncthreads_and(tc_mbar_wait(tc_smem_u32(&mbar[pb]), phase[pb])) != 0;
      if (!ok) break;   // block-uniform; the drain below waits again with a limit
      phase[pb] ^= 1u;
      tc_fence_after();
      flush(pb);
    }
  }
  if (ok && nch > 0) {
    const int lb = (nch - 1) & 1;
    ok = __syncthreads_and(tc_mbar_wait(tc_smem_u32(&mbar[lb]), phase[lb])) != 0;
    if (ok) {
      tc_fence_after();
      flush(lb);
    }
  }
  if (!ok) {
    // drain: every committed chunk completes before the tensor memory goes
    for (int b = 0; b < 2; ++b) (void)__syncthreads_and(tc_mbar_wait(tc_smem_u32(&mbar[b]), phase[b]));
    if (tid == 0) atomicCAS(status, 0, (int)QTT_ETIMEOUT);
  } else {
    // lane r = 32 (warp % 4) + lane: element (i0 + r / 2), component r % 2;
    // adjacent lanes write the two floats of one complex value
    const int r = 32 * (warp & 3) + (tid & 31);
    const long long i = i0 + (r >> 1);
    const int comp = r & 1;
    float* Cf;
    long long sCi, sCj;
    if (part) {
      Cf = reinterpret_cast<float*>(part + (long long)split * ldpart);
      sCi = 1;
      sCj = g.M;
    } else {
      Cf = reinterpret_cast<float*>(g.C + g.bC1 * b1 + g.bC2 * b2);
      sCi = g.sCi;
      sCj = g.sCj;
    }
    if (i < g.M) {
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const long long j = j0 + 32 * half + q;
        if (j < g.N) Cf[2 * (i * sCi + j * sCj) + comp] = sum[q] - cmp[q];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)TC_TCOLS)
                 : "memory");
}

static std::atomic<unsigned long long> g_tc_cfg[2];

template <typename TA>
qtt_status tc_cgemm(const CGemmArgs<TA>& g, int nbatch, int* status, cudaStream_t s,
                    const char* name) {
  if (g.M <= 0 || g.N <= 0 || nbatch <= 0) return QTT_OK;
  if (!status || g.nb1 < 1 || nbatch > 65535 || (g.M + 63) / 64 > 65535) {
    set_error("tc_cgemm: bad shape, batch or status word");
    return QTT_EINVAL;
  }
  if (first_on_device(&g_tc_cfg[sizeof(TA) == sizeof(float) ? 0 : 1]))
    cudaFuncSetAttribute(k_tc_cgemm<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  const long long tiles = (long long)((g.N + TN_TC - 1) / TN_TC) * ((g.M + 63) / 64);
  const int sms = device_sm_count();
  int splits = 1;
  if (nbatch == 1) {
    // split k beyond TC_KMAX terms per CTA, and further while the tiles
    // alone cannot fill the GPU (runs of at least 4 chunks)
    splits = (g.K + TC_KMAX - 1) / TC_KMAX;
    if (tiles * splits < 2LL * sms)
      splits = (int)std::max<long long>(
          splits, std::min<long long>((2LL * sms + tiles - 1) / tiles, (long long)g.K / (4 * TC_KC)));
    splits = std::max(1, std::min(splits, 64));
  }
  const int kchunk = std::max(TC_KC, ((g.K + splits - 1) / splits + TC_KC - 1) / TC_KC * TC_KC);
  splits = std::max(1, (g.K + kchunk - 1) / kchunk);   // no empty split
  dim3 grid((unsigned)((g.N + TN_TC - 1) / TN_TC), (unsigned)((g.M + 63) / 64),
            (unsigned)(nbatch * splits));
  QTT_PROF(name, s);
  const double mnk = (double)g.M * g.N * g.K * nbatch;
  prof_add_work(name, (sizeof(TA) == sizeof(float) ? 4.0 : 8.0) * mnk,
                ((double)g.M * g.K * sizeof(TA) + (double)g.K * g.N * 8.0 + (double)g.M * g.N * 8.0) *
                    nbatch);
  if (splits == 1) {
    k_tc_cgemm<TA><<<grid, TC_THREADS, TC_SMEM, s>>>(g, nbatch, kchunk, nullptr, 0, status);
    return QTT_OK;
  }
  const long long ldpart = (long long)g.M * g.N;
  float2* part = (float2*)scratch_alloc(sizeof(float2) * (size_t)(ldpart * splits), s);
  if (!part) {
    set_error("tc_cgemm: split-k scratch allocation failed");
    return QTT_ENOMEM;
  }
  k_tc_cgemm<TA><<<grid, TC_THREADS, TC_SMEM, s>>>(g, 1, kchunk, part, ldpart, status);
  cgemm_reduce(part, splits, ldpart, g.M, g.N, g.C, g.sCi, g.sCj, s);
  scratch_free(part, s);
  return QTT_OK;
}
template qtt_status tc_cgemm<float>(const CGemmArgs<float>&, int, int*, cudaStream_t, const char*);
template qtt_status tc_cgemm<float2>(const CGemmArgs<float2>&, int, int*, cudaStream_t, const char*);

// which kernel the large-rank rounding's products use.  0 (default): the
// CUDA-core GEMM with compensated chunk sums.  The tensor cores' FP32
// accumulator rounds one-signed, and along the range finder's chain of
// products that bias reaches the result (measured on the exact-regime
// 256 x 256 case: E2 3e-5 against < 1e-5); 1 selects them anyway.
static int g_tc_gemm = 0;
int tc_gemm_enabled() { return g_tc_gemm; }

}  // namespace qtt

extern "C" void qtt_debug_set_tc_gemm(int on) { qtt::g_tc_gemm = (on == 1 || on == 2) ? on : 0; }

// C (M x N, column-major, complex64) = op(A) B through the tensor-core GEMM:
// A (M x K, column-major, complex64; conjugated when conjA), B (K x N,
// column-major).  *status_dev receives QTT_ETIMEOUT if a wait ran out.
extern "C" qtt_status qtt_debug_tc_cgemm(const void* A, const void* B, void* C, int M, int N, int K,
                                         int conjA, int* status_dev, void* stream) {
  clear_error();
  if (M < 0 || N < 0 || K < 0 || !status_dev || (!A && M > 0 && K > 0) ||
      (!B && K > 0 && N > 0) || (!C && M > 0 && N > 0)) {
    set_error("qtt_debug_tc_cgemm: NULL argument or negative size");
    return QTT_EINVAL;
  }
  if (M == 0 || N == 0) return QTT_OK;
  qtt::CGemmArgs<float2> g;
  g.A = (const float2*)A; g.sAi = 1; g.sAk = M;
  g.B = (const float2*)B; g.sBk = 1; g.sBj = K;
  g.C = (float2*)C; g.sCi = 1; g.sCj = M;
  g.M = M; g.N = N; g.K = K; g.conjA = conjA;
  if (K == 0) {
    const qtt_status st = qtt::cuda_check(
        cudaMemsetAsync(C, 0, sizeof(float2) * (size_t)M * N, (cudaStream_t)stream), "tc_cgemm");
    return st;
  }
  const qtt_status st = qtt::tc_cgemm<float2>(g, 1, status_dev, (cudaStream_t)stream, "tc_cgemm");
  if (st != QTT_OK) return st;
  return qtt::cuda_check(cudaGetLastError(), "tc_cgemm launch");
}

namespace qtt {

// ---------------------------------------------------------------------------
// Gram partials on the tensor cores: for X (m x n complex64, column-major,
// ld m, m = m_mul * *m_ptr <= mp) every CTA sums G = X X^H over its columns
// and writes it to gram_part[blockIdx.x] (ldp x ldp, element (a, b) at
// a + ldp b, zero outside m x m) -- the partial format of the CUDA-core
// Gram pass, reduced in FP64 by the same reduction.
//
// Real form: with Y = [Re X | Im X] and Z = [Im X | -Re X] (real k 2j, 2j+1
// = column j), Y Y^T = Re G and Z Y^T = Im G, since
// Im(x conj(y)) = Im x Re y - Re x Im y.  A chunk is 8 complex columns (two
// TF32 k-steps of 8).  When 2 mp <= 128 one M = 128 MMA takes the stacked
// [Y; Z] as A and Y (its first mp rows) as B (N = mp); above, two MMAs put
// Re G in tensor-memory columns 0.. and Im G in 128.. .  SPLIT = 1 feeds
// each value rounded to TF32 (one product per k-step: the first pass of the
// TF32-refined TT-SVD, whose second pass recomputes the Gram in FP32);
// SPLIT = 3 feeds hi + lo (3xTF32).
constexpr int TG_THREADS = 256;
constexpr int TG_KC = 8;                       // complex columns per chunk
constexpr int TG_TILE = 128 * 8 * 4;           // one 128-row TF32 k-step tile
constexpr int TG_BUF = 8 * TG_TILE;            // {Y, Z} x {hi, lo} x two k-steps
// requested dynamic shared memory: two buffers, and at least 80 KB so that
// at most two CTAs share an SM (each holds 256 tensor-memory columns)
constexpr size_t TG_SMEM = (2 * (size_t)TG_BUF + 1024) > 80 * 1024 ? (2 * (size_t)TG_BUF + 1024)
                                                                   : 80 * 1024;

__device__ __forceinline__ unsigned char* tg_tile(unsigned char* buf, int op, int part, int step) {
  return buf + (size_t)(((op * 2 + part) * 2 + step)) * TG_TILE;
}

__device__ __forceinline__ void tg_put4(unsigned char* buf, int op, int step, int row, int kq,
                                        float4 v, bool split) {
  const uint32_t off = tc_tile_off(row, 4 * kq);
  float4 hi = make_float4(tc_tf32(v.x), tc_tf32(v.y), tc_tf32(v.z), tc_tf32(v.w));
  *reinterpret_cast<float4*>(tg_tile(buf, op, 0, step) + off) = hi;
  if (split) {
    float4 lo = make_float4(tc_tf32(v.x - hi.x), tc_tf32(v.y - hi.y), tc_tf32(v.z - hi.z),
                            tc_tf32(v.w - hi.w));
    *reinterpret_cast<float4*>(tg_tile(buf, op, 1, step) + off) = lo;
  }
}

template <int SPLIT>
__global__ void __launch_bounds__(TG_THREADS, 1)
k_tc_gram(const float2* __restrict__ X, const int* __restrict__ m_ptr, int m_mul, long long n,
          int mp, float2* __restrict__ gram_part, int ldp, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char tg_dyn[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  constexpr bool split = (SPLIT == 3);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m = min(m_mul * (*m_ptr), mp);
  const bool single = (2 * mp <= 128);
  unsigned char* base = tg_dyn + ((1024u - (tc_smem_u32(tg_dyn) & 1023u)) & 1023u);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc_smem_u32(&tmem_slot)),
                 "r"(256u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    tc_mbar_init(tc_smem_u32(&mbar[0]), 1);
    tc_mbar_init(tc_smem_u32(&mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = tc_idesc_tf32(128, mp);

  // this thread's (row, column pair) slots of a chunk: mp rows x 4 pairs
  const int nslot = mp * 4;
  constexpr int TG_MAXS = 128 * 4 / TG_THREADS;   // 2
  const long long nchunk = (n + TG_KC - 1) / TG_KC;
  const int my = (blockIdx.x < nchunk) ? (int)((nchunk - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  float2 r0[TG_MAXS], r1[TG_MAXS];
  auto load_chunk = [&](int c) {
    const long long j0 = (blockIdx.x + (long long)c * gridDim.x) * TG_KC;
#pragma unroll
    for (int t = 0; t < TG_MAXS; ++t) {
      const int e = tid + t * TG_THREADS;
      const int a = e % mp, g = e / mp;
      const long long j = j0 + 2 * g;
      const bool ok = (e < nslot) && (a < m);
      r0[t] = (ok && j < n) ? __ldg(X + a + (long long)m * j) : make_float2(0.f, 0.f);
      r1[t] = (ok && j + 1 < n) ? __ldg(X + a + (long long)m * (j + 1)) : make_float2(0.f, 0.f);
    }
  };
  uint32_t phase[2] = {0u, 0u};
  int used[2] = {0, 0};
  bool ok = true;
  if (my > 0) load_chunk(0);
  for (int c = 0; c < my; ++c) {
    const int buf = c & 1;
    unsigned char* sb = base + (size_t)buf * TG_BUF;
    if (used[buf]) {
      ok = __syncthreads_and(tc_mbar_wait(tc_smem_u32(&mbar[buf]), phase[buf])) != 0;
      if (!ok) break;
      phase[buf] ^= 1u;
      used[buf] = 0;
    }
#pragma unroll
    for (int t = 0; t < TG_MAXS; ++t) {
      const int e = tid + t * TG_THREADS;
      if (e < nslot) {
        const int a = e % mp, g = e / mp;
        const int step = g >> 1, kq = g & 1;
        const float2 x0 = r0[t], x1 = r1[t];
        tg_put4(sb, 0, step, a, kq, make_float4(x0.x, x0.y, x1.x, x1.y), split);
        if (single)
          tg_put4(sb, 0, step, mp + a, kq, make_float4(x0.y, -x0.x, x1.y, -x1.x), split);
        else
          tg_put4(sb, 1, step, a, kq, make_float4(x0.y, -x0.x, x1.y, -x1.x), split);
      }
    }
    tc_fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int step = 0; step < 2; ++step) {
        const uint32_t acc0 = (c > 0 || step > 0) ? 1u : 0u;
        const uint64_t yh = tc_sdesc(tc_smem_u32(tg_tile(sb, 0, 0, step)), TC_LBO, TC_SBO);
        const uint64_t yl = tc_sdesc(tc_smem_u32(tg_tile(sb, 0, 1, step)), TC_LBO, TC_SBO);
        if (single) {
          tc_mma_tf32(tmem, yh, yh, idesc, acc0);
          if (split) {
            tc_mma_tf32(tmem, yh, yl, idesc, 1u);
            tc_mma_tf32(tmem, yl, yh, idesc, 1u);
          }
        } else {
          const uint64_t zh = tc_sdesc(tc_smem_u32(tg_tile(sb, 1, 0, step)), TC_LBO, TC_SBO);
          const uint64_t zl = tc_sdesc(tc_smem_u32(tg_tile(sb, 1, 1, step)), TC_LBO, TC_SBO);
          tc_mma_tf32(tmem, yh, yh, idesc, acc0);
          tc_mma_tf32(tmem + 128, zh, yh, idesc, acc0);
          if (split) {
            tc_mma_tf32(tmem, yh, yl, idesc, 1u);
            tc_mma_tf32(tmem, yl, yh, idesc, 1u);
            tc_mma_tf32(tmem + 128, zh, yl, idesc, 1u);
            tc_mma_tf32(tmem + 128, zl, yh, idesc, 1u);
          }
        }
      }
      tc_commit(tc_smem_u32(&mbar[buf]));
    }
    used[buf] = 1;
    if (c + 1 < my) load_chunk(c + 1);
  }
#pragma unroll
  for (int b = 0; b < 2; ++b)
    if (used[b]) {
      if (!__syncthreads_and(tc_mbar_wait(tc_smem_u32(&mbar[b]), phase[b]))) ok = false;
      phase[b] ^= 1u;
    }
  tc_fence_after();
  __syncthreads();
  float2* gp = gram_part + (size_t)blockIdx.x * ldp * ldp;
  float* gpf = reinterpret_cast<float*>(gp);
  // entries outside the mp x mp block covered by the MMAs
  for (int e = tid; e < ldp * ldp; e += TG_THREADS) {
    const int a = e % ldp, b = e / ldp;
    if (a >= mp || b >= mp) gp[e] = make_float2(0.f, 0.f);
  }
  if (!ok) {
    if (tid == 0) atomicCAS(status, 0, (int)QTT_ETIMEOUT);
  } else {
    const int lane = 32 * (warp & 3) + (tid & 31);
    const int half = warp >> 2;
    const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
    // single: lanes < mp hold Re G rows, lanes mp.. 2 mp Im G rows;
    // double: lanes are rows, columns 0.. Re, 128.. Im
    const int nrep = single ? 1 : 2;
    for (int rep = 0; rep < nrep; ++rep) {
      int a, comp;
      if (single) { a = lane < mp ? lane : lane - mp; comp = lane < mp ? 0 : 1; }
      else { a = lane; comp = rep; }
      const bool live = single ? (lane < 2 * mp) : (lane < mp);
      for (int p = half; p < mp / 16; p += 2) {
        float v[16];
        if (my > 0) {
          tc_ld16(tmem + lane_addr + (uint32_t)(128 * rep + 16 * p), v);
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q) v[q] = 0.f;
        }
        if (live && a < ldp) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int b = 16 * p + q;
            if (b < ldp) gpf[2 * (a + (size_t)ldp * b) + comp] = v[q];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u)
                 : "memory");
}

static std::atomic<unsigned long long> g_tg_cfg[2];

int tc_gram(const float2* X, const int* m_ptr, int m_mul, int mcap, long long n, int split,
            float2* gram_part, int ldp, int max_parts, int* status, cudaStream_t s) {
  const int mp = std::max(16, (mcap + 15) / 16 * 16);
  const long long nchunk = (n + TG_KC - 1) / TG_KC;
  int grid = (int)std::min<long long>(std::max<long long>(nchunk, 1), (long long)max_parts);
  if (grid < 1) grid = 1;
  QTT_PROF(split == 3 ? "tc_gram_3xtf32" : "tc_gram_tf32", s);
  // algorithmic work: the m x n complex operand once; m^2 n complex MACs
  prof_add_work(split == 3 ? "tc_gram_3xtf32" : "tc_gram_tf32", 8.0 * mcap * (double)mcap * n,
                8.0 * mcap * (double)n);
  if (split == 3) {
    if (first_on_device(&g_tg_cfg[1]))
      cudaFuncSetAttribute(k_tc_gram<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TG_SMEM);
    k_tc_gram<3><<<grid, TG_THREADS, TG_SMEM, s>>>(X, m_ptr, m_mul, n, mp, gram_part, ldp, status);
  } else {
    if (first_on_device(&g_tg_cfg[0]))
      cudaFuncSetAttribute(k_tc_gram<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TG_SMEM);
    k_tc_gram<1><<<grid, TG_THREADS, TG_SMEM, s>>>(X, m_ptr, m_mul, n, mp, gram_part, ldp, status);
  }
  return grid;
}

}  // namespace qtt

// Gram partials of X (m x n complex64, column-major) on the tensor cores:
// gram_part (nparts x ldp x ldp complex64) as the TT-SVD's first pass
// computes them; returns nparts (<= max_parts), or a negative status.
extern "C" int qtt_debug_tc_gram(const void* X, int m, long long n, int split, void* gram_part,
                                 int ldp, int max_parts, int* status_dev, void* stream) {
  clear_error();
  if (!X || !gram_part || !status_dev || m < 1 || m > 128 || n < 0 || ldp < m || ldp > 128 ||
      max_parts < 1 || (split != 1 && split != 3)) {
    set_error("qtt_debug_tc_gram: bad argument");
    return QTT_EINVAL;
  }
  int* mdev = nullptr;
  if (cudaMallocAsync(&mdev, sizeof(int), (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    set_error("qtt_debug_tc_gram: allocation failed");
    return QTT_ENOMEM;
  }
  cudaMemcpyAsync(mdev, &m, sizeof(int), cudaMemcpyHostToDevice, (cudaStream_t)stream);
  const int np = qtt::tc_gram((const float2*)X, mdev, 1, m, n, split, (float2*)gram_part, ldp,
                              max_parts, status_dev, (cudaStream_t)stream);
  cudaFreeAsync(mdev, (cudaStream_t)stream);
  const qtt_status st = qtt::cuda_check(cudaGetLastError(), "tc_gram launch");
  return st == QTT_OK ? np : (int)st;
}
