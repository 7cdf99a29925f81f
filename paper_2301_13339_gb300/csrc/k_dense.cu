// Dense building blocks of the large-rank rounding (ranks above 64):
//
//  * big_qr_q  -- blocked Householder QR of an m x n matrix held in global
//    memory (m <= BQ_MAXM) and the formation of the first nq columns of Q.
//    Panels of BQ_NB columns are factored by one CTA in shared memory
//    (LAPACK's H_k = I - tau_k v_k v_k^H, v_k = [1; A[k+1:, k]]), their
//    compact-WY factor T (H_1 ... H_nb = I - V T V^H, upper triangular) is
//    formed in the same CTA, and the trailing columns are updated with
//    Q^H = I - V T^H V^H by many CTAs (8 columns each).  Q = H_1 ... H_k
//    [I; 0] is then accumulated panel by panel from the last one.  Householder
//    QR keeps Q orthonormal to working precision also when A is rank
//    deficient, which the randomised range finder of the rounding needs.
//
//  * cgemm      -- C = op(A) B for complex64 B and C and a complex64 or real
//    A, any strides (unit stride along the rows of A or along k; along k for
//    B; along the rows of C), batched over a two-level batch index.  64 x 64
//    output tiles, 16-deep k chunks staged in shared memory, 4 x 4 outputs
//    per thread; each chunk is summed with plain FMAs and added to the
//    running sum with compensation (Kahan), so long contractions keep
//    about one rounding error per chunk instead of one per term.
#include "qtt_internal.cuh"
#include "house_qr.cuh"
#include <algorithm>
#include <atomic>

namespace qtt {

// ---------------------------------------------------------------- QR
constexpr int BQ_NB = 32;        // panel width
constexpr int BQ_THREADS = 512;  // panel CTA
constexpr int BQ_CB = 8;         // columns per CTA in the block-reflector application
constexpr int BQ_MAXM = 768;     // rows (panel in shared memory: 768 x 32 x 8 B)

// A[k:, j] <- (I - t v v^H) A[k:, j] with v = [1; A[k+1:, k]] (rows of P, ld
// mp); one warp.
template <typename T>
__device__ __forceinline__ void bq_apply_col(T* P, int mp, int k, T t, int j) {
  const int lane = threadIdx.x & 31;
  const T* vk = P + (size_t)mp * k;
  T* x = P + (size_t)mp * j;
  T w = szero<T>();
  for (int i = k + lane; i < mp; i += 32) {
    const T v = (i == k) ? sone(T()) : vk[i];
    macc(w, v, x[i]);
  }
  w = warp_sum(w);
  const T f = smul(t, w);
  for (int i = k + lane; i < mp; i += 32) {
    const T v = (i == k) ? sone(T()) : vk[i];
    x[i] = ssub(x[i], smul(v, f));
  }
}

// Factor the panel A[p:m, p:p+kb] (kb <= BQ_NB) in shared memory, write it
// back (R on and above the diagonal, the v_k below) and T (BQ_NB x BQ_NB,
// column-major) to Tm.
template <typename T>
__global__ void __launch_bounds__(BQ_THREADS)
k_bq_panel(T* __restrict__ A, int m, int p, int kb, T* __restrict__ Tm) {
  extern __shared__ __align__(16) unsigned char bq_smem[];
  T* P = reinterpret_cast<T*>(bq_smem);
  __shared__ T s_tau[BQ_NB];
  __shared__ T s_Y[BQ_NB * BQ_NB];
  __shared__ T s_T[BQ_NB * BQ_NB];
  const int mp = m - p;
  const int tid = threadIdx.x, warp = tid >> 5, nw = BQ_THREADS / 32;
  for (int e = tid; e < mp * kb; e += BQ_THREADS) {
    const int i = e % mp, j = e / mp;
    P[e] = A[(size_t)(p + i) + (size_t)m * (p + j)];
  }
  for (int e = tid; e < BQ_NB * BQ_NB; e += BQ_THREADS) {
    s_T[e] = szero<T>();
    s_Y[e] = szero<T>();
  }
  __syncthreads();
  const int kmax = min(mp, kb);
  if (kmax > 0 && warp == 0) house_form_reflector(P, mp, 0, s_tau);
  __syncthreads();
  for (int k = 0; k < kmax; ++k) {
    const T ctau = conjg(s_tau[k]);
    if (warp == 0) {
      if (k + 1 < kb) {
        bq_apply_col(P, mp, k, ctau, k + 1);
        __syncwarp();
        if (k + 1 < kmax) house_form_reflector(P, mp, k + 1, s_tau);
      }
    } else {
      for (int j = k + 2 + (warp - 1); j < kb; j += nw - 1) bq_apply_col(P, mp, k, ctau, j);
    }
    __syncthreads();
  }
  // Y[a + NB b] = v_a^H v_b (a < b), one warp per pair
  for (int pr = warp; pr < kmax * kmax; pr += nw) {
    const int a = pr % kmax, b = pr / kmax;
    if (a >= b) continue;
    const int lane = tid & 31;
    T acc = szero<T>();
    for (int i = b + lane; i < mp; i += 32) {
      const T vb = (i == b) ? sone(T()) : P[i + (size_t)mp * b];
      macc(acc, P[i + (size_t)mp * a], vb);   // i >= b > a: v_a[i] = P[i, a]
    }
    acc = warp_sum(acc);
    if (lane == 0) s_Y[a + BQ_NB * b] = acc;
  }
  __syncthreads();
  // T(b, b) = tau_b;  T(0:b, b) = -tau_b T(0:b, 0:b) Y(0:b, b)
  if (warp == 0) {
    const int lane = tid & 31;
    for (int b = 0; b < kmax; ++b) {
      T val = szero<T>();
      if (lane < b) {
        for (int c = lane; c < b; ++c) mac(val, s_T[lane + BQ_NB * c], s_Y[c + BQ_NB * b]);
        val = smul(make_scalar<T>(-sreal(s_tau[b]), -simag(s_tau[b])), val);
      }
      __syncwarp();
      if (lane < b) s_T[lane + BQ_NB * b] = val;
      if (lane == b) s_T[b + BQ_NB * b] = s_tau[b];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = tid; e < mp * kb; e += BQ_THREADS) {
    const int i = e % mp, j = e / mp;
    A[(size_t)(p + i) + (size_t)m * (p + j)] = P[e];
  }
  for (int e = tid; e < BQ_NB * BQ_NB; e += BQ_THREADS) Tm[e] = s_T[e];
}

// X[p:m, c] <- (I - V op(T) V^H) X[p:m, c] for the columns c of this CTA
// (col0 + BQ_CB blockIdx.x + [0, BQ_CB), below col0 + ncols); V = the kb
// reflectors stored in A[p:m, p:p+kb] (unit diagonal).  adj = 1: op(T) = T^H
// (applies Q^H, the trailing update); adj = 0: op(T) = T (forms Q).
template <typename T>
__global__ void __launch_bounds__(256)
k_bq_apply(T* X, int m, int col0, int ncols, const T* A, int p, int kb, const T* __restrict__ Tm,
           int adj) {
  __shared__ T Vs[32][BQ_NB + 1];
  __shared__ T Xs[32][BQ_CB];
  __shared__ T W[BQ_NB][BQ_CB];
  __shared__ T W2[BQ_NB][BQ_CB];
  const int tid = threadIdx.x;
  const int cbase = col0 + BQ_CB * blockIdx.x;
  const int mp = m - p;
  const int a = tid % BQ_NB, c = tid / BQ_NB;   // 32 x 8
  T acc = szero<T>();
  for (int r0 = 0; r0 < mp; r0 += 32) {
    __syncthreads();
    for (int e = tid; e < 32 * BQ_NB; e += 256) {
      const int ri = e % 32, aa = e / 32, i = r0 + ri;
      T v = szero<T>();
      if (i < mp && aa < kb) v = (i == aa) ? sone(T()) : (i > aa) ? A[(size_t)(p + i) + (size_t)m * (p + aa)] : szero<T>();
      Vs[ri][aa] = v;
    }
    {
      const int ri = tid % 32, cc = tid / 32, i = r0 + ri;
      const int col = cbase + cc;
      Xs[ri][cc] = (i < mp && col < col0 + ncols) ? X[(size_t)(p + i) + (size_t)m * col] : szero<T>();
    }
    __syncthreads();
    const int rn = min(32, mp - r0);
    for (int ri = 0; ri < rn; ++ri) macc(acc, Vs[ri][a], Xs[ri][c]);
  }
  W[a][c] = acc;
  __syncthreads();
  {
    T w2 = szero<T>();
    if (a < kb) {
      if (adj) {
        for (int b = 0; b <= a; ++b) macc(w2, Tm[b + BQ_NB * a], W[b][c]);   // conj(T[b, a])
      } else {
        for (int b = a; b < kb; ++b) mac(w2, Tm[a + BQ_NB * b], W[b][c]);
      }
    }
    W2[a][c] = w2;
  }
  for (int r0 = 0; r0 < mp; r0 += 32) {
    __syncthreads();
    for (int e = tid; e < 32 * BQ_NB; e += 256) {
      const int ri = e % 32, aa = e / 32, i = r0 + ri;
      T v = szero<T>();
      if (i < mp && aa < kb) v = (i == aa) ? sone(T()) : (i > aa) ? A[(size_t)(p + i) + (size_t)m * (p + aa)] : szero<T>();
      Vs[ri][aa] = v;
    }
    __syncthreads();
    const int ri = tid % 32, cc = tid / 32, i = r0 + ri;
    const int col = cbase + cc;
    if (i < mp && col < col0 + ncols) {
      T s = szero<T>();
      for (int aa = 0; aa < kb; ++aa) mac(s, Vs[ri][aa], W2[aa][cc]);
      T* xp = X + (size_t)(p + i) + (size_t)m * col;
      *xp = ssub(*xp, s);
    }
  }
}

// Q[i + m j] = (i == j), j < nq
template <typename T>
__global__ void k_bq_eye(T* Q, int m, int nq) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)m * nq) return;
  const int i = (int)(e % m), j = (int)(e / m);
  Q[e] = (i == j) ? sone(T()) : szero<T>();
}

// A[i + m j] = conj(S[j + ls i])  (A = S^H, m x n, from S n x m)
template <typename T>
__global__ void k_conj_transpose(const T* S, int ls, int n, int m, T* A) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)m * n) return;
  const int i = (int)(e % m), j = (int)(e / m);
  A[e] = conjg(S[j + (size_t)ls * i]);
}

size_t big_qr_panel_smem(int m) { return sizeof(float2) * (size_t)m * BQ_NB; }
size_t big_qr_tm_elems(int n) { return (size_t)((n + BQ_NB - 1) / BQ_NB) * BQ_NB * BQ_NB; }

static std::atomic<unsigned long long> g_bq_cfg[2];

template <typename T>
static void bq_configure() {
  if (first_on_device(&g_bq_cfg[sizeof(T) == sizeof(double) ? 1 : 0]))
    cudaFuncSetAttribute(k_bq_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(T) * BQ_MAXM * BQ_NB));
}

template <typename T>
qtt_status big_qr_q(T* A, int m, int n, int nq, T* Q, T* Tm, cudaStream_t s) {
  if (m < 1 || n < 1 || nq < 1 || m > BQ_MAXM || nq > m) {
    set_error("big_qr: shape %d x %d (nq %d) outside the supported range (m <= %d)", m, n, nq,
              BQ_MAXM);
    return QTT_EINVAL;
  }
  bq_configure<T>();
  const int kmax = std::min(m, n);
  for (int p = 0; p < kmax; p += BQ_NB) {
    const int kb = std::min(BQ_NB, kmax - p);
    T* Tp = Tm + (size_t)(p / BQ_NB) * BQ_NB * BQ_NB;
    {
      QTT_PROF("bigqr_panel", s);
      k_bq_panel<T><<<1, BQ_THREADS, sizeof(T) * (size_t)(m - p) * kb, s>>>(A, m, p, kb, Tp);
    }
    const int c0 = p + kb, nc = kmax - c0;
    if (nc > 0) {
      QTT_PROF("bigqr_update", s);
      k_bq_apply<T><<<(nc + BQ_CB - 1) / BQ_CB, 256, 0, s>>>(A, m, c0, nc, A, p, kb, Tp, 1);
    }
  }
  {
    QTT_PROF("bigqr_formq", s);
    k_bq_eye<T><<<(unsigned)(((long long)m * nq + 255) / 256), 256, 0, s>>>(Q, m, nq);
  }
  const int np = (kmax + BQ_NB - 1) / BQ_NB;
  for (int pi = np - 1; pi >= 0; --pi) {
    const int p = pi * BQ_NB;
    const int kb = std::min(BQ_NB, kmax - p);
    if (p >= nq) continue;
    QTT_PROF("bigqr_formq", s);
    k_bq_apply<T><<<(nq - p + BQ_CB - 1) / BQ_CB, 256, 0, s>>>(
        Q, m, p, nq - p, A, p, kb, Tm + (size_t)pi * BQ_NB * BQ_NB, 0);
  }
  return cuda_check(cudaGetLastError(), "big_qr launch");
}
template qtt_status big_qr_q<float2>(float2*, int, int, int, float2*, float2*, cudaStream_t);
template qtt_status big_qr_q<double>(double*, int, int, int, double*, double*, cudaStream_t);

template <typename T>
void launch_conj_transpose(const T* S, int ls, int n, int m, T* A, cudaStream_t s) {
  k_conj_transpose<T><<<(unsigned)(((long long)m * n + 255) / 256), 256, 0, s>>>(S, ls, n, m, A);
}
template void launch_conj_transpose<float2>(const float2*, int, int, int, float2*, cudaStream_t);
template void launch_conj_transpose<double>(const double*, int, int, int, double*, cudaStream_t);

// ---------------------------------------------------------------- GEMM
constexpr int CG_BM = 64, CG_BN = 64, CG_BK = 16, CG_THREADS = 256;

__device__ __forceinline__ void cg_mac(float2& acc, float a, float2 b) {
  acc.x = fmaf(a, b.x, acc.x);
  acc.y = fmaf(a, b.y, acc.y);
}
__device__ __forceinline__ void cg_mac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ float cg_conj(float a) { return a; }
__device__ __forceinline__ float2 cg_conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float cg_zero(float) { return 0.f; }
__device__ __forceinline__ float2 cg_zero(float2) { return make_float2(0.f, 0.f); }
// Kahan: s + c carries the sum; add v
__device__ __forceinline__ void cg_kadd(float2& s, float2& c, float2 v) {
  float y = v.x - c.x, t = s.x + y;
  c.x = (t - s.x) - y;
  s.x = t;
  y = v.y - c.y;
  t = s.y + y;
  c.y = (t - s.y) - y;
  s.y = t;
}

template <typename TA>
__global__ void __launch_bounds__(CG_THREADS) k_cgemm(CGemmArgs<TA> g) {
  __shared__ TA As[CG_BK][CG_BM + 1];
  __shared__ float2 Bs[CG_BK][CG_BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int bz = blockIdx.z;
  const int b1 = bz % g.nb1, b2 = bz / g.nb1;
  const TA* A = g.A + g.bA1 * b1 + g.bA2 * b2;
  const float2* B = g.B + g.bB1 * b1 + g.bB2 * b2;
  float2* C = g.C + g.bC1 * b1 + g.bC2 * b2;
  const long long i0 = (long long)blockIdx.y * CG_BM, j0 = (long long)blockIdx.x * CG_BN;
  float2 sum[4][4], cmp[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      sum[u][v] = make_float2(0.f, 0.f);
      cmp[u][v] = make_float2(0.f, 0.f);
    }
  const bool a_rows_unit = (g.sAi == 1);
  for (int k0 = 0; k0 < g.K; k0 += CG_BK) {
    __syncthreads();
    for (int e = tid; e < CG_BM * CG_BK; e += CG_THREADS) {
      int ii, kk;
      if (a_rows_unit) { ii = e % CG_BM; kk = e / CG_BM; }
      else { kk = e % CG_BK; ii = e / CG_BK; }
      const long long i = i0 + ii;
      const int k = k0 + kk;
      TA v = cg_zero(TA());
      if (i < g.M && k < g.K) {
        v = A[i * g.sAi + (long long)k * g.sAk];
        if (g.conjA) v = cg_conj(v);
      }
      As[kk][ii] = v;
    }
    for (int e = tid; e < CG_BN * CG_BK; e += CG_THREADS) {
      const int kk = e % CG_BK, jj = e / CG_BK;
      const long long j = j0 + jj;
      const int k = k0 + kk;
      Bs[kk][jj] = (j < g.N && k < g.K) ? B[(long long)k * g.sBk + j * g.sBj] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 part[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) part[u][v] = make_float2(0.f, 0.f);
#pragma unroll
    for (int kk = 0; kk < CG_BK; ++kk) {
      TA a[4];
      float2 b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[kk][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Bs[kk][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) cg_mac(part[u][v], a[u], b[v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) cg_kadd(sum[u][v], cmp[u][v], part[u][v]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const long long i = i0 + ty + 16 * u;
    if (i >= g.M) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const long long j = j0 + tx + 16 * v;
      if (j >= g.N) continue;
      C[i * g.sCi + j * g.sCj] = make_float2(sum[u][v].x - cmp[u][v].x, sum[u][v].y - cmp[u][v].y);
    }
  }
}

template <typename TA>
qtt_status cgemm(const CGemmArgs<TA>& g, int nbatch, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || nbatch <= 0) return QTT_OK;
  if (g.nb1 < 1 || nbatch > 65535) {
    set_error("cgemm: bad batch (%d, nb1 %d)", nbatch, g.nb1);
    return QTT_EINVAL;
  }
  dim3 grid((unsigned)((g.N + CG_BN - 1) / CG_BN), (unsigned)((g.M + CG_BM - 1) / CG_BM),
            (unsigned)nbatch);
  if (grid.y > 65535) {
    set_error("cgemm: M = %d too large", g.M);
    return QTT_EINVAL;
  }
  QTT_PROF("round_gemm", s);
  const double mnk = (double)g.M * g.N * g.K * nbatch;
  prof_add_work("round_gemm", (sizeof(TA) == sizeof(float) ? 4.0 : 8.0) * mnk,
                ((double)g.M * g.K * sizeof(TA) + (double)g.K * g.N * 8.0 + (double)g.M * g.N * 8.0) *
                    nbatch);
  k_cgemm<TA><<<grid, CG_THREADS, 0, s>>>(g);
  return QTT_OK;
}
template qtt_status cgemm<float>(const CGemmArgs<float>&, int, cudaStream_t);
template qtt_status cgemm<float2>(const CGemmArgs<float2>&, int, cudaStream_t);

}  // namespace qtt
