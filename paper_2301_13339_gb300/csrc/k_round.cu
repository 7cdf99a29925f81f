// TT-rounding of the operator x vector product Y = O X (the convolution step
// of Alg. 2 done with the QTT Toeplitz operator), without forming Y.
//
// Y_k[(a + r_{k-1} p), j, (b + r_k q)] = sum_i O_k[p, j, i, q] X_k[a, i, b]
// has ranks R_k = P_k r_k (about 16 x 64).  Textbook rounding (QR sweep, then
// truncated-SVD sweep) would factor R_k x 2 R_k matrices.  Instead:
//   1. left sketch   WL_k = Omega_{<=k}^T Y_{<=k}  (l_k x R_k) for a Gaussian
//                    TT Omega of ranks l_k (counter-based Philox4x32-10
//                    generator, Salmon et al. 2011), computed core by core
//                    through the factors O_k and X_k;
//   2. right-to-left Z = Y_k C_k (R_{k-1} x 2 l'_k); an orthonormal basis
//                    V of the row space of the sketch WL_{k-1} Z becomes the
//                    right-orthonormal core Q_k = V^H, C_{k-1} = Z V
//                    (randomised range finder per cut: the TT is now right-
//                    orthonormal with ranks l' <= sketch);
//   3. left-to-right truncated SVD sweep on that TT with the threshold rule
//                    of Alg. 1 (tau = eps/sqrt(d-1) ||Y||) and the rank cap:
//                    the deterministic rounding step.
// All factorisations are Gram + Jacobi (+ refinement) on <= 128 x 128.
#include "qtt_internal.cuh"
#include "house_qr.cuh"
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <atomic>

namespace qtt {

// ---------------------------------------------------------------- Philox
__host__ __device__ inline void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n1 = lo1;
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  uint32_t n3 = lo0;
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}
__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  uint32_t k[2] = {k0, k1};
  for (int r = 0; r < 10; ++r) {
    philox_round(c, k);
    k[0] += 0x9E3779B9u;
    k[1] += 0xBB67AE85u;
  }
}

// out[e] ~ N(0, 1), e < n; counter = (e, core, 0, 0), key = seed.
template <typename R>
__global__ void gauss_fill_kernel(R* out, long long n, unsigned long long seed, uint32_t core) {
  const long long e2 = ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  if (2 * e2 >= n) return;
  uint32_t c[4] = {(uint32_t)e2, (uint32_t)(e2 >> 32), core, 0x51ca7u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u1 = ((double)c[0] + 0.5) * 2.3283064365386963e-10;
  const double u2 = ((double)c[1] + 0.5) * 2.3283064365386963e-10;
  const double rad = sqrt(-2.0 * log(u1));
  out[2 * e2] = (R)(rad * cospi(2.0 * u2));
  if (2 * e2 + 1 < n) out[2 * e2 + 1] = (R)(rad * sinpi(2.0 * u2));
}

#define GRID1(n) (unsigned)(((n) + 255) / 256), 256, 0, s

void launch_gauss_fill(float* out, long long n, unsigned long long seed, uint32_t tag, cudaStream_t s) {
  gauss_fill_kernel<float><<<(unsigned)((n / 2 + 1 + 255) / 256), 256, 0, s>>>(out, n, seed, tag);
}
void launch_gauss_fill(double* out, long long n, unsigned long long seed, uint32_t tag, cudaStream_t s) {
  gauss_fill_kernel<double><<<(unsigned)((n / 2 + 1 + 255) / 256), 256, 0, s>>>(out, n, seed, tag);
}

// Orthonormal sketch cores.  Each Gaussian core Omega_k, read as the
// (2 l_{k-1}) x l_k matrix Om[s' + l0 (j + 2 s)] (l_k <= 2 l_{k-1}), is
// replaced by the Q factor of its Gram-Schmidt orthonormalisation (classical
// Gram-Schmidt applied twice per column).  The left sketch Omega_{<=k} then
// has orthonormal columns: a random isometry of the 2^k-dimensional left
// space, exactly an orthogonal change of basis at cuts where l_k = 2^k.  With
// plain Gaussian cores the TT sketch's condition number grows with k, and in
// FP32 that loses digits in the range finder of step 2.
constexpr int OS_THREADS = 256;
constexpr int OS_MAXD = 32;
struct SketchCores {
  long long off[OS_MAXD];
  int m[OS_MAXD];   // 2 l_{k-1}
  int n[OS_MAXD];   // l_k
};
template <typename R>
__global__ void __launch_bounds__(OS_THREADS) k_orth_sketch(R* Om, SketchCores sc) {
  extern __shared__ __align__(16) unsigned char os_smem[];
  R* M = reinterpret_cast<R*>(os_smem);
  __shared__ R s_c[128];
  __shared__ R s_red[OS_THREADS / 32];
  const int k = blockIdx.x + 1;
  const int m = sc.m[k], n = sc.n[k];
  R* G = Om + sc.off[k];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = OS_THREADS / 32;
  for (int e = tid; e < m * n; e += OS_THREADS) M[e] = G[e];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    R* v = M + (size_t)m * j;
    for (int pass = 0; pass < 2; ++pass) {
      // c_i = <M_i, v> for i < j: one warp per coefficient
      for (int i = warp; i < j; i += nw) {
        const R* qi = M + (size_t)m * i;
        R a = 0;
        for (int r = lane; r < m; r += 32) a += qi[r] * v[r];
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) s_c[i] = a;
      }
      __syncthreads();
      for (int r = tid; r < m; r += OS_THREADS) {
        R a = v[r];
        for (int i = 0; i < j; ++i) a -= s_c[i] * M[r + (size_t)m * i];
        v[r] = a;
      }
      __syncthreads();
    }
    R a = 0;
    for (int r = tid; r < m; r += OS_THREADS) a += v[r] * v[r];
    for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    if (lane == 0) s_red[warp] = a;
    __syncthreads();
    R nrm2 = 0;
    for (int w = 0; w < nw; ++w) nrm2 += s_red[w];
    const R inv = nrm2 > (R)0 ? (R)1 / sqrt(nrm2) : (R)0;
    for (int r = tid; r < m; r += OS_THREADS) v[r] *= inv;
    __syncthreads();
  }
  for (int e = tid; e < m * n; e += OS_THREADS) G[e] = M[e];
}

// The contractions below are one output per thread, summed in index order
// with compensation; their operands come from L2, so the loops load KB
// terms ahead (independent loads in flight) and then add them in the same
// order as a plain loop would.
constexpr int KB = 8;

// ---------------------------------------------------------------- step 1
// A1[s + lk (j + 2 c)] = sum_{s'} Om[s' + l0 (j + 2 s)] WL0[s' + l0 c],  c < R0
template <typename T, typename R>
__global__ void k_a1(const R* Om, int l0, int lk, const T* WL0, const int* xr, int k, int Pin,
                     int Rc0, T* A1) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int R0 = Pin * xr[k - 1];
  if (e >= (long long)lk * 2 * Rc0) return;
  const int s = (int)(e % lk), j = (int)((e / lk) % 2), c = (int)(e / (2LL * lk));
  if (c >= R0) return;
  typename KAccOf<T>::type acc;
  const R* om = Om + (size_t)l0 * (j + 2 * s);
  const T* wl = WL0 + (size_t)l0 * c;
  for (int s0 = 0; s0 < l0; s0 += KB) {
    R o[KB];
    T w[KB];
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      o[t] = (s0 + t < l0) ? om[s0 + t] : (R)0;
      w[t] = (s0 + t < l0) ? wl[s0 + t] : szero<T>();
    }
#pragma unroll
    for (int t = 0; t < KB; ++t)
      if (s0 + t < l0) acc.add_rmul(o[t], w[t]);
  }
  A1[s + (size_t)lk * (j + 2 * c)] = acc.get();
}
// A2[s + lk (j + 2 (p + Pin (i + 2 b)))] = sum_a A1[s + lk (j + 2 (a + r0 p))] X[a + r0 (i + 2 b)]
template <typename T>
__global__ void k_a2(const T* A1, int lk, const T* X, const int* xr, int k, int Pin, int rcap1,
                     T* A2) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r0 = xr[k - 1], r1 = xr[k];
  if (e >= (long long)lk * 2 * Pin * 2 * rcap1) return;
  const int s = (int)(e % lk);
  long long t = e / lk;
  const int j = (int)(t % 2); t /= 2;
  const int p = (int)(t % Pin); t /= Pin;
  const int i = (int)(t % 2); t /= 2;
  const int b = (int)t;
  if (b >= r1) return;
  typename KAccOf<T>::type acc;
  for (int a0 = 0; a0 < r0; a0 += KB) {
    T x1[KB], x2[KB];
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      const int a = a0 + t;
      x1[t] = (a < r0) ? A1[s + (size_t)lk * (j + 2 * (a + r0 * p))] : szero<T>();
      x2[t] = (a < r0) ? X[a + (size_t)r0 * (i + 2 * b)] : szero<T>();
    }
#pragma unroll
    for (int t = 0; t < KB; ++t)
      if (a0 + t < r0) acc.add_mul(x1[t], x2[t]);
  }
  A2[s + (size_t)lk * (j + 2 * (p + Pin * (i + 2 * b)))] = acc.get();
}
// WL1[s + lk (b + r1 q)] = sum_{j,p,i} O[p + Pin (j + 2 (i + 2 q))] A2[s + lk (j + 2 (p + Pin (i + 2 b)))]
template <typename T, typename R>
__global__ void k_wl(const R* O, int Pin, int Pout, const T* A2, int lk, const int* xr, int k,
                     int Rc1, T* WL1) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r1 = xr[k];
  if (e >= (long long)lk * Rc1) return;
  const int s = (int)(e % lk), c = (int)(e / lk);
  if (c >= Pout * r1) return;
  const int b = c % r1, q = c / r1;
  typename KAccOf<T>::type acc;
  // terms (i, p, j) in that nesting order, flattened: f = j + 2 (p + Pin i)
  const int nf = 4 * Pin;
  for (int f0 = 0; f0 < nf; f0 += KB) {
    R o[KB];
    T x[KB];
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      const int f = f0 + t;
      const int j = f & 1, p = (f >> 1) % Pin, i = (f >> 1) / Pin;
      o[t] = (f < nf) ? O[p + Pin * (j + 2 * (i + 2 * q))] : (R)0;
      x[t] = (f < nf) ? A2[s + (size_t)lk * (j + 2 * (p + Pin * (i + 2 * b)))] : szero<T>();
    }
#pragma unroll
    for (int t = 0; t < KB; ++t)
      if (o[t] != (R)0) acc.add_rmul(o[t], x[t]);
  }
  WL1[s + (size_t)lk * c] = acc.get();
}

// In-place scaling of a sketch block to unit max-abs entry.  The
// sketch of Y_{<=k} grows like (sqrt(l) ||Y_k||)^k; any scaling of a sketch
// leaves its row space unchanged, so each WL_k is rescaled as it is formed.
// Over many CTAs: the largest |entry| (non-negative floats compare as their
// bit patterns) by atomicMax into *mx (zeroed before), then the division by
// it.
template <typename T>
__global__ void k_absmax(const T* A, int lk, const int* xr, int k, int Pout, unsigned* mx) {
  const long long n = (long long)lk * Pout * xr[k];
  float m = 0.f;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, sqrtf((float)sabs2(A[e])));
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, __float_as_uint(m));
}
template <typename T>
__global__ void k_scale_max(T* A, int lk, const int* xr, int k, int Pout, const unsigned* mx) {
  const float m = __uint_as_float(*mx);
  if (!(m > 0.f) || !(m < 3.0e38f)) return;
  const long long n = (long long)lk * Pout * xr[k];
  const typename Sc<T>::R sc = (typename Sc<T>::R)(1.0 / (double)m);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    A[e] = rscale(A[e], sc);
}

// ---------------------------------------------------------------- QR
// One-CTA Householder QR of A = S^H (m x nc, m = rows of the basis, nc <= 64)
// read from S (nc x m, ld ls); writes the first nq columns of Q (m x nq, ld m)
// with orthonormal columns spanning the row space of S (Householder QR is
// backward stable and keeps Q orthonormal also when S is rank deficient).
// The factorisation and the formation of Q are in house_qr.cuh.
template <typename T>
__global__ void __launch_bounds__(QR_THREADS)
k_house_q(const T* __restrict__ S, int ls, int m, int nc, int nq, T* __restrict__ Q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);      // m x nc, ld m
  T* E = A + (size_t)m * nc;                  // m x nq, ld m
  __shared__ T s_tau[128];
  for (int e = threadIdx.x; e < m * nc; e += QR_THREADS) {
    const int i = e % m, j = e / m;
    A[e] = conjg(S[j + (size_t)ls * i]);
  }
  __syncthreads();
  const int kmax = min(m, nc);
  house_qr_factor(A, m, nc, s_tau);
  house_form_q(A, m, kmax, nq, s_tau, E);
  for (int e = threadIdx.x; e < m * nq; e += QR_THREADS) Q[e] = E[e];
}

// ---------------------------------------------------------------- step 2
// B1[a + r0 (i + 2 (q + Pout t))] = sum_b X[a + r0 (i + 2 b)] C[(b + r1 q) + ldc t]
template <typename T>
__global__ void k_b1(const T* X, const int* xr, int k, int rcap0, int Pout, const T* C, int ldc,
                     int lq, int d, T* B1) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r0 = xr[k - 1], r1 = xr[k];
  if (e >= (long long)rcap0 * 2 * Pout * lq) return;
  const int a = (int)(e % rcap0);
  long long t = e / rcap0;
  const int i = (int)(t % 2); t /= 2;
  const int q = (int)(t % Pout); t /= Pout;
  const int tt = (int)t;
  if (a >= r0) return;
  typename KAccOf<T>::type acc;
  for (int b0 = 0; b0 < r1; b0 += KB) {
    T x1[KB], x2[KB];
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      const int b = b0 + t;
      x1[t] = (b < r1) ? X[a + (size_t)r0 * (i + 2 * b)] : szero<T>();
      x2[t] = (b < r1) ? C[(b + r1 * q) + (size_t)ldc * tt] : szero<T>();
    }
#pragma unroll
    for (int t = 0; t < KB; ++t)
      if (b0 + t < r1) acc.add_mul(x1[t], x2[t]);
  }
  B1[a + (size_t)r0 * (i + 2 * (q + Pout * tt))] = acc.get();
}
// Z[(a + r0 p) + ldz (j + 2 t)] = sum_{q,i} O[p + Pin (j + 2 (i + 2 q))] B1[a + r0 (i + 2 (q + Pout t))]
template <typename T, typename R>
__global__ void k_z(const R* O, int Pin, int Pout, const T* B1, const int* xr, int k, int rcap0,
                    int lq, int ldz, T* Z) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r0 = xr[k - 1];
  if (e >= (long long)rcap0 * Pin * 2 * lq) return;
  const int a = (int)(e % rcap0);
  long long t = e / rcap0;
  const int p = (int)(t % Pin); t /= Pin;
  const int j = (int)(t % 2); t /= 2;
  const int tt = (int)t;
  if (a >= r0) return;
  typename KAccOf<T>::type acc;
  // terms (q, i) in that nesting order, flattened: f = i + 2 q
  const int nf = 2 * Pout;
  for (int f0 = 0; f0 < nf; f0 += KB) {
    R o[KB];
    T x[KB];
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      const int f = f0 + t;
      const int i = f & 1, q = f >> 1;
      o[t] = (f < nf) ? O[p + Pin * (j + 2 * (i + 2 * q))] : (R)0;
      x[t] = (f < nf) ? B1[a + (size_t)r0 * (i + 2 * (q + Pout * tt))] : szero<T>();
    }
#pragma unroll
    for (int t = 0; t < KB; ++t)
      if (o[t] != (R)0) acc.add_rmul(o[t], x[t]);
  }
  Z[(a + r0 * p) + (size_t)ldz * (j + 2 * tt)] = acc.get();
}
// S[s + l0 u] = sum_{c < R0} WL[s + l0 c] Z[c + ldz u]  (R0 = P r up to ~1e3):
// KS_SPLIT threads share one output, each a compensated partial sum over
// every KS_SPLIT-th c, combined by shuffles within the group
constexpr int KS_SPLIT = 8;
template <typename T>
__global__ void k_s(const T* WL, int l0, const T* Z, int ldz, const int* xr, int k, int Pin,
                    int ncolu, T* S) {
  const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  const long long e = g / KS_SPLIT;
  const int part = (int)(g % KS_SPLIT);
  const bool live = e < (long long)l0 * ncolu;
  const int R0 = Pin * xr[k - 1];
  typename KAccOf<T>::type acc;
  if (live) {
    const int s = (int)(e % l0), u = (int)(e / l0);
    for (int c0 = part; c0 < R0; c0 += KB * KS_SPLIT) {
      T x1[KB], x2[KB];
#pragma unroll
      for (int t = 0; t < KB; ++t) {
        const int c = c0 + t * KS_SPLIT;
        x1[t] = (c < R0) ? WL[s + (size_t)l0 * c] : szero<T>();
        x2[t] = (c < R0) ? Z[c + (size_t)ldz * u] : szero<T>();
      }
#pragma unroll
      for (int t = 0; t < KB; ++t)
        if (c0 + t * KS_SPLIT < R0) acc.add_mul(x1[t], x2[t]);
    }
  }
  T v = acc.get();
  // groups of KS_SPLIT consecutive lanes (blockDim is a multiple of 32)
  for (int off = 1; off < KS_SPLIT; off <<= 1) v = sadd(v, shfl_xor_s(v, off));
  if (live && part == 0) S[e] = v;
}
// column Gram  G[u + ldg v] = sum_s conj(S[s + ls u]) S[s + ls v],  u, v < n (rows ls)
template <typename T>
__global__ void k_gram_cols(const T* S, int ls, int n, double2* G, int ldg) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int u = e % n, v = e / n;
  typename KAccOf<T>::type acc;
  for (int q0 = 0; q0 < ls; q0 += KB) {
    T x1[KB], x2[KB];
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      const int s2 = q0 + t;
      x1[t] = (s2 < ls) ? S[s2 + (size_t)ls * u] : szero<T>();
      x2[t] = (s2 < ls) ? S[s2 + (size_t)ls * v] : szero<T>();
    }
#pragma unroll
    for (int t = 0; t < KB; ++t)
      if (q0 + t < ls) acc.add_cmul(x1[t], x2[t]);
  }
  G[u + (size_t)ldg * v] = to_d2(acc.get());
}
// SV[s + ls w] = sum_u S[s + ls u] V[u + n w]
template <typename T>
__global__ void k_sv(const T* S, int ls, int n, const T* V, T* SV) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ls * n) return;
  const int s2 = e % ls, w = e / ls;
  typename KAccOf<T>::type acc;
  for (int u0 = 0; u0 < n; u0 += KB) {
    T x1[KB], x2[KB];
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      const int u = u0 + t;
      x1[t] = (u < n) ? S[s2 + (size_t)ls * u] : szero<T>();
      x2[t] = (u < n) ? V[u + (size_t)n * w] : szero<T>();
    }
#pragma unroll
    for (int t = 0; t < KB; ++t)
      if (u0 + t < n) acc.add_mul(x1[t], x2[t]);
  }
  SV[e] = acc.get();
}
// Q[s + lq0 (j + 2 t)] = conj(V[(j + 2 t) + n s]),  n = 2 lq
template <typename T>
__global__ void k_qcore(const T* V, int n, int lq0, T* Q) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= lq0 * n) return;
  const int s2 = e % lq0, u = e / lq0;
  Q[e] = conjg(V[u + (size_t)n * s2]);
}
// Cn[c + ldc s] = sum_u Z[c + ldz u] V[u + n s],  c < R0
template <typename T>
__global__ void k_c(const T* Z, int ldz, const T* V, int n, int lq0, const int* xr, int k, int Pin,
                    int ldc, T* Cn) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)ldc * lq0) return;
  const int c = (int)(e % ldc), s2 = (int)(e / ldc);
  if (c >= Pin * xr[k - 1]) return;
  typename KAccOf<T>::type acc;
  for (int u0 = 0; u0 < n; u0 += KB) {
    T x1[KB], x2[KB];
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      const int u = u0 + t;
      x1[t] = (u < n) ? Z[c + (size_t)ldz * u] : szero<T>();
      x2[t] = (u < n) ? V[u + (size_t)n * s2] : szero<T>();
    }
#pragma unroll
    for (int t = 0; t < KB; ++t)
      if (u0 + t < n) acc.add_mul(x1[t], x2[t]);
  }
  Cn[c + (size_t)ldc * s2] = acc.get();
}

// ---------------------------------------------------------------- step 3
// Zt[(s + t0 j) + m u] = sum_{s' < lq0} Lc[s + t0 s'] Tp[s' + lq0 (j + 2 u)],  m = 2 t0
template <typename T>
__global__ void k_zt(const T* Lc, const int* tr, int k, int tcap0, const T* Tp, int lq0, int lq,
                     T* Zt) {
  const int t0 = tr[k - 1];
  const int m = 2 * t0;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * tcap0 * lq) return;
  const int row = e % (2 * tcap0), u = e / (2 * tcap0);
  if (row >= m) return;
  const int s2 = row % t0, j = row / t0;
  typename KAccOf<T>::type acc;
  for (int q0 = 0; q0 < lq0; q0 += KB) {
    T x1[KB], x2[KB];
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      const int sp = q0 + t;
      x1[t] = (sp < lq0) ? Lc[s2 + (size_t)t0 * sp] : szero<T>();
      x2[t] = (sp < lq0) ? Tp[sp + (size_t)lq0 * (j + 2 * u)] : szero<T>();
    }
#pragma unroll
    for (int t = 0; t < KB; ++t)
      if (q0 + t < lq0) acc.add_mul(x1[t], x2[t]);
  }
  Zt[row + (size_t)m * u] = acc.get();
}
// row Gram  G[a + ldg b] = sum_u Z[a + m u] conj(Z[b + m u]),  m = mul * *mptr
template <typename T>
__global__ void k_gram_rows(const T* Zt, const int* mptr, int mul, int mcap, int ncol, double2* G,
                            int ldg) {
  const int m = mul * (*mptr);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= mcap * mcap) return;
  const int a = e % mcap, b = e / mcap;
  if (a >= m || b >= m) return;
  typename KAccOf<T>::type acc;
  for (int u0 = 0; u0 < ncol; u0 += KB) {
    T x1[KB], x2[KB];
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      const int u = u0 + t;
      x1[t] = (u < ncol) ? Zt[b + (size_t)m * u] : szero<T>();
      x2[t] = (u < ncol) ? Zt[a + (size_t)m * u] : szero<T>();
    }
#pragma unroll
    for (int t = 0; t < KB; ++t)
      if (u0 + t < ncol) acc.add_cmul(x1[t], x2[t]);
  }
  G[a + (size_t)ldg * b] = to_d2(acc.get());
}
// W[c + m u] = sum_a conj(U[a + m c]) Z[a + m u],  c < rows (= rmul * *rptr or m)
template <typename T>
__global__ void k_proj_rows(const T* U, const T* Zt, const int* mptr, int mul, const int* rptr,
                            int mcap, int ncol, T* W) {
  const int m = mul * (*mptr);
  const int rr = rptr ? *rptr : m;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= mcap * ncol) return;
  const int c = e % mcap, u = e / mcap;
  if (c >= rr) return;
  typename KAccOf<T>::type acc;
  for (int a0 = 0; a0 < m; a0 += KB) {
    T x1[KB], x2[KB];
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      const int a = a0 + t;
      x1[t] = (a < m) ? U[a + (size_t)m * c] : szero<T>();
      x2[t] = (a < m) ? Zt[a + (size_t)m * u] : szero<T>();
    }
#pragma unroll
    for (int t = 0; t < KB; ++t)
      if (a0 + t < m) acc.add_cmul(x1[t], x2[t]);
  }
  W[c + (size_t)rr * u] = acc.get();
}
// Step 3 with more rows than columns (m = 2 t_{k-1} > lq_k): Zt = Q R by
// Householder (one CTA) first, so the rank decision factors the
// lq_k x lq_k Gram of R instead of the m x m Gram of Zt (whose rank is at
// most lq_k).  Q: m x kk (ld m), R: kk x nc (ld kk), kk = min(m, nc) also
// written to *kdev for the kernels that follow.
template <typename T>
__global__ void __launch_bounds__(QR_THREADS)
k_qr_rows(const T* __restrict__ Zt, const int* mptr, int mul, int nc, T* __restrict__ Q,
          T* __restrict__ R, int* kdev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T s_tau[128];
  const int m = mul * (*mptr);
  const int kk = min(m, nc);
  T* A = reinterpret_cast<T*>(smem_raw);     // m x nc
  T* E = A + (size_t)m * nc;                 // m x kk
  for (int e = threadIdx.x; e < m * nc; e += QR_THREADS) A[e] = Zt[e];
  __syncthreads();
  house_qr_factor(A, m, nc, s_tau);
  for (int e = threadIdx.x; e < kk * nc; e += QR_THREADS) {
    const int i = e % kk, j = e / kk;
    R[e] = (i <= j) ? A[i + (size_t)m * j] : szero<T>();
  }
  house_form_q(A, m, kk, kk, s_tau, E);
  for (int e = threadIdx.x; e < m * kk; e += QR_THREADS) Q[e] = E[e];
  if (threadIdx.x == 0) *kdev = kk;
}
// core[i + m c] = sum_a Q[i + m a] Ur[a + kk c],  i < m = 2 t_{k-1}, c < r_k
template <typename T>
__global__ void k_qu(const T* Q, const int* mptr, const int* kdev, const T* Ur, const int* rptr,
                     int mcap, int rcap, T* core) {
  const int m = 2 * (*mptr), kk = *kdev, r = *rptr;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= mcap * rcap) return;
  const int i = e % mcap, c = e / mcap;
  if (i >= m || c >= r) return;
  typename KAccOf<T>::type acc;
  for (int a = 0; a < kk; ++a) acc.add_mul(Q[i + (size_t)m * a], Ur[a + (size_t)kk * c]);
  core[i + (size_t)m * c] = acc.get();
}

__global__ void k_one(void* p, int is_f64) {
  if (threadIdx.x == 0) {
    if (is_f64) *(double*)p = 1.0;
    else *(float2*)p = make_float2(1.f, 0.f);
  }
}
__global__ void k_set_ranks_one(int* r, int d) {
  if (threadIdx.x == 0) { r[0] = 1; r[d] = 1; }
}

// ---------------------------------------------------------------- sketch cache
// The orthonormalised sketch cores are a function of (device, element type,
// seed, l profile) only, so they are generated once per key and kept (up to
// SK_CACHE_MAX bytes in total; beyond that, or while the stream is being
// captured into a CUDA graph, a miss generates them into per-call scratch).
// A new entry is complete before it is returned (one wait per key), so any
// stream or graph may use it.
struct SketchEntry {
  void* ptr = nullptr;
  cudaEvent_t ev = nullptr;
  bool ready = false;
  size_t bytes = 0;
};
typedef std::tuple<int, int, unsigned long long, std::vector<int>> SketchKey;
static std::mutex g_sk_mu;
static std::map<SketchKey, SketchEntry> g_sk_cache;
static size_t g_sk_bytes = 0;
constexpr size_t SK_CACHE_MAX = (size_t)64 << 20;

void sketch_cache_clear() {
  std::lock_guard<std::mutex> lk(g_sk_mu);
  for (auto& kv : g_sk_cache) {
    if (kv.second.ptr) cudaFree(kv.second.ptr);
    if (kv.second.ev) cudaEventDestroy(kv.second.ev);
  }
  g_sk_cache.clear();
  g_sk_bytes = 0;
}

// real <-> complex copies of one sketch core for the blocked QR
template <typename R>
__global__ void k_real_to_c(const R* a, long long n, float2* b) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) b[e] = make_float2((float)a[e], 0.f);
}
template <typename R>
__global__ void k_c_to_real(const float2* b, long long n, R* a) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) a[e] = (R)b[e].x;
}

static std::atomic<unsigned long long> g_os_cfg[2];

// Cores of at most OS_MAX_ELEMS elements are orthonormalised by Gram-Schmidt
// in one launch (one CTA each); larger ones (ranks above 64) by the blocked
// Householder QR, one after the other.
constexpr int OS_MAX_ELEMS = 128 * 64;

template <typename R>
static qtt_status generate_sketch(R* Om, const std::vector<int>& l, const std::vector<size_t>& omoff,
                                  int d, unsigned long long seed, cudaStream_t s) {
  for (int k = 1; k < d; ++k) {
    const long long n = (long long)l[k - 1] * 2 * l[k];
    QTT_PROF("round_sketch", s);
    gauss_fill_kernel<R><<<(unsigned)((n / 2 + 1 + 255) / 256), 256, 0, s>>>(Om + omoff[k], n, seed,
                                                                              (uint32_t)k);
  }
  if (d <= 1) return QTT_OK;
  SketchCores sc{};
  int mmax = 1;
  std::vector<int> big;
  for (int k = 1; k < d && k < OS_MAXD; ++k) {
    sc.off[k] = (long long)omoff[k];
    const int m = 2 * l[k - 1], n = l[k];
    if (m * n > OS_MAX_ELEMS) {
      big.push_back(k);
      sc.m[k] = 0;
      sc.n[k] = 0;
      continue;
    }
    sc.m[k] = m;
    sc.n[k] = n;
    mmax = std::max(mmax, m * n);
  }
  if (first_on_device(&g_os_cfg[sizeof(R) == sizeof(double) ? 1 : 0]))
    cudaFuncSetAttribute(k_orth_sketch<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(R) * OS_MAX_ELEMS));
  {
    QTT_PROF("round_sketch", s);
    k_orth_sketch<R><<<d - 1, OS_THREADS, sizeof(R) * (size_t)mmax, s>>>(Om, sc);
  }
  if (big.empty()) return QTT_OK;
  // blocked QR of each large core, through complex copies
  size_t emax = 0;
  int nmax = 1;
  for (int k : big) {
    emax = std::max(emax, (size_t)2 * l[k - 1] * l[k]);
    nmax = std::max(nmax, l[k]);
  }
  float2* Ac = (float2*)scratch_alloc(sizeof(float2) * emax, s);
  float2* Qc = (float2*)scratch_alloc(sizeof(float2) * emax, s);
  float2* Tm = (float2*)scratch_alloc(sizeof(float2) * big_qr_tm_elems(nmax), s);
  qtt_status st = QTT_OK;
  if (!Ac || !Qc || !Tm) {
    set_error("round: sketch scratch allocation failed");
    st = QTT_ENOMEM;
  }
  for (size_t b = 0; b < big.size() && st == QTT_OK; ++b) {
    const int k = big[b];
    const int m = 2 * l[k - 1], n = l[k];
    const long long e = (long long)m * n;
    QTT_PROF("round_sketch", s);
    k_real_to_c<R><<<(unsigned)((e + 255) / 256), 256, 0, s>>>(Om + omoff[k], e, Ac);
    st = big_qr_q<float2>(Ac, m, n, n, Qc, Tm, s);
    if (st == QTT_OK) k_c_to_real<R><<<(unsigned)((e + 255) / 256), 256, 0, s>>>(Qc, e, Om + omoff[k]);
  }
  scratch_free(Ac, s);
  scratch_free(Qc, s);
  scratch_free(Tm, s);
  return st;
}

// Returns the sketch cores for (seed, l); *owned = true when the caller must
// scratch_free them after use.
template <typename R>
static R* get_sketch(const std::vector<int>& l, const std::vector<size_t>& omoff, size_t omtot,
                     int d, unsigned long long seed, cudaStream_t s, bool* owned) {
  int dev = 0;
  cudaGetDevice(&dev);
  SketchKey key(dev, (int)sizeof(R), seed, l);
  const size_t bytes = sizeof(R) * std::max<size_t>(omtot, 1);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  {
    std::lock_guard<std::mutex> lk(g_sk_mu);
    auto it = g_sk_cache.find(key);
    if (it != g_sk_cache.end()) {
      *owned = false;
      return (R*)it->second.ptr;
    }
    if (cs == cudaStreamCaptureStatusNone && g_sk_bytes + bytes <= SK_CACHE_MAX) {
      SketchEntry en;
      if (cudaMalloc(&en.ptr, bytes) == cudaSuccess &&
          cudaEventCreateWithFlags(&en.ev, cudaEventDisableTiming) == cudaSuccess) {
        const qtt_status gst = generate_sketch<R>((R*)en.ptr, l, omoff, d, seed, s);
        // complete before any stream (or graph) can use the entry
        cudaEventRecord(en.ev, s);
        cudaEventSynchronize(en.ev);
        if (gst != QTT_OK) {
          cudaFree(en.ptr);
          cudaEventDestroy(en.ev);
          return nullptr;
        }
        en.ready = true;
        en.bytes = bytes;
        g_sk_bytes += bytes;
        g_sk_cache[key] = en;
        *owned = false;
        return (R*)en.ptr;
      }
      cudaGetLastError();
      if (en.ptr) cudaFree(en.ptr);
    }
  }
  R* Om = (R*)scratch_alloc(bytes, s);
  if (!Om) return nullptr;
  if (generate_sketch<R>(Om, l, omoff, d, seed, s) != QTT_OK) {
    scratch_free(Om, s);
    return nullptr;
  }
  *owned = true;
  return Om;
}

template <typename T>
static qtt_status round_product_t(const qtt_op* op, const qtt_tensor* x, const qtt_trunc& tr,
                                  int sketch, unsigned long long seed, cudaStream_t s,
                                  qtt_tensor** out) {
  using R = typename Sc<T>::R;
  const int d = x->desc.d;
  const bool refine = tr.refine || !Sc<T>::cplx;
  if (sketch <= 0) sketch = QTT_RANK_CAP;
  sketch = std::min(sketch, QTT_RANK_CAP);
  const int rmax_eff = std::min(tr.rmax > 0 ? tr.rmax : QTT_RANK_CAP, QTT_RANK_CAP);
  // forced ranks (parity mode): the cap-only rule with a per-cut cap
  const int* fixed = tr.fixed_ranks;
  auto cap_at = [&](int k) { return fixed ? std::min(fixed[k], QTT_RANK_CAP) : rmax_eff; };
  const double eps_u = fixed ? 0.0 : tr.eps;
  const double delta_u = fixed ? 0.0 : tr.delta;
  const std::vector<int>& P = op->P;
  const std::vector<int>& xcap = x->rcap;
  std::vector<int> Rc(d + 1), l(d + 1), lq(d + 1), ocap(d + 1);
  for (int k = 0; k <= d; ++k) Rc[k] = P[k] * xcap[k];
  for (int k = 0; k <= d; ++k) {
    long long lim = std::min<long long>(1LL << std::min(k, 40), 1LL << std::min(d - k, 40));
    l[k] = (int)std::min<long long>({(long long)sketch, lim, (long long)Rc[k]});
  }
  l[0] = l[d] = 1;
  // the left sketch at cut k spans at most 2 l_{k-1} directions
  for (int k = 1; k < d; ++k) l[k] = std::min(l[k], 2 * l[k - 1]);
  lq[d] = 1;
  for (int k = d; k >= 2; --k) lq[k - 1] = std::min(l[k - 1], 2 * lq[k]);
  lq[0] = 1;
  ocap[0] = 1;
  for (int k = 1; k < d; ++k) ocap[k] = std::min({2 * ocap[k - 1], lq[k], cap_at(k)});
  ocap[d] = 1;

  const R* Oc = (const R*)op->cores;
  const T* Xc = (const T*)x->cores;
  // --- buffers
  int Rmax = 1, lmax = 1;
  for (int k = 0; k <= d; ++k) { Rmax = std::max(Rmax, Rc[k]); lmax = std::max(lmax, l[k]); }
  int Pmax = 1, xmax = 1;
  for (int k = 0; k <= d; ++k) { Pmax = std::max(Pmax, P[k]); xmax = std::max(xmax, xcap[k]); }
  std::vector<size_t> wloff(d);
  size_t wltot = 0;
  for (int k = 0; k < d; ++k) { wloff[k] = wltot; wltot += (size_t)l[k] * Rc[k]; }
  std::vector<size_t> omoff(d);
  size_t omtot = 0;
  for (int k = 1; k < d; ++k) { omoff[k] = omtot; omtot += (size_t)l[k - 1] * 2 * l[k]; }
  T* WL = (T*)scratch_alloc(sizeof(T) * std::max<size_t>(wltot, 1), s);
  bool om_owned = false;
  R* Om = get_sketch<R>(l, omoff, omtot, d, seed, s, &om_owned);
  const size_t a1sz = (size_t)lmax * 2 * Rmax;
  const size_t a2sz = (size_t)lmax * 2 * Pmax * 2 * xmax;
  T* A1 = (T*)scratch_alloc(sizeof(T) * a1sz, s);
  T* A2 = (T*)scratch_alloc(sizeof(T) * std::max(a2sz, (size_t)xmax * 2 * Pmax * 64), s);
  T* Z = (T*)scratch_alloc(sizeof(T) * (size_t)Rmax * 2 * 64, s);
  T* C0 = (T*)scratch_alloc(sizeof(T) * (size_t)Rmax * 64, s);
  T* C1 = (T*)scratch_alloc(sizeof(T) * (size_t)Rmax * 64, s);
  T* S = (T*)scratch_alloc(sizeof(T) * 64 * 128, s);
  T* SV = (T*)scratch_alloc(sizeof(T) * 128 * 128, s);
  T* SV2 = (T*)scratch_alloc(sizeof(T) * 128 * 128, s);
  T* V1 = (T*)scratch_alloc(sizeof(T) * 128 * 128, s);
  T* V = (T*)scratch_alloc(sizeof(T) * 128 * 128, s);
  double2* G = (double2*)scratch_alloc(sizeof(double2) * 128 * 128, s);
  T* Zt = (T*)scratch_alloc(sizeof(T) * 128 * 64, s);
  T* W1 = (T*)scratch_alloc(sizeof(T) * 128 * 64, s);
  T* Lc = (T*)scratch_alloc(sizeof(T) * 64 * 64, s);
  T* one = (T*)scratch_alloc(sizeof(T), s);
  T* Qz = (T*)scratch_alloc(sizeof(T) * 128 * 64, s);
  T* Rz = (T*)scratch_alloc(sizeof(T) * 64 * 64, s);
  T* Ur = (T*)scratch_alloc(sizeof(T) * 64 * 64, s);
  int* kd = (int*)scratch_alloc(sizeof(int), s);
  unsigned* wmax = (unsigned*)scratch_alloc(sizeof(unsigned) * (d + 1), s);
  // every scratch buffer goes back to the pool on every exit
  auto release = [&]() {
    scratch_free(WL, s); if (om_owned) scratch_free(Om, s); scratch_free(A1, s); scratch_free(A2, s);
    scratch_free(Z, s); scratch_free(C0, s); scratch_free(C1, s); scratch_free(S, s);
    scratch_free(SV, s); scratch_free(SV2, s); scratch_free(V1, s); scratch_free(V, s);
    scratch_free(G, s); scratch_free(Zt, s); scratch_free(W1, s); scratch_free(Lc, s);
    scratch_free(one, s); scratch_free(Qz, s); scratch_free(Rz, s); scratch_free(Ur, s);
    scratch_free(kd, s); scratch_free(wmax, s);
  };
  if (!WL || !Om || !A1 || !A2 || !Z || !C0 || !C1 || !S || !SV || !SV2 || !V1 || !V || !G || !Zt ||
      !W1 || !Lc || !one || !Qz || !Rz || !Ur || !kd || !wmax) {
    release();
    set_error("round: scratch allocation failed");
    return QTT_ENOMEM;
  }
  const int is64 = Sc<T>::cplx ? 0 : 1;
  k_one<<<1, 32, 0, s>>>(one, is64);
  cudaMemsetAsync(wmax, 0, sizeof(unsigned) * (d + 1), s);
  // intermediate right-orthonormal TT (host-known ranks lq)
  TensorDesc pd = x->desc;
  qtt_tensor* Tp = nullptr;
  qtt_status st = tensor_alloc(pd, lq, s, &Tp);
  if (st != QTT_OK) { release(); return st; }
  T* Tpc = (T*)Tp->cores;
  // output
  qtt_tensor* y = nullptr;
  st = tensor_alloc(x->desc, ocap, s, &y);
  if (st != QTT_OK) { tensor_free_async(Tp, s); release(); return st; }
  k_set_ranks_one<<<1, 32, 0, s>>>(y->ranks, d);

  // --- 1. left sketches through the (cached) orthonormal sketch cores
  cudaMemcpyAsync(WL + wloff[0], one, sizeof(T), cudaMemcpyDeviceToDevice, s);
  for (int k = 1; k < d; ++k) {
    const int l0 = l[k - 1], lk = l[k];
    const R* Ok = Oc + op->off[k - 1];
    const T* Xk = Xc + x->off[k - 1];
    { QTT_PROF("round_sketch", s);
    k_a1<T, R><<<GRID1((long long)lk * 2 * Rc[k - 1])>>>(Om + omoff[k], l0, lk, WL + wloff[k - 1],
                                                         x->ranks, k, P[k - 1], Rc[k - 1], A1);
    }
    { QTT_PROF("round_sketch", s);
    k_a2<T><<<GRID1((long long)lk * 2 * P[k - 1] * 2 * xcap[k])>>>(A1, lk, Xk, x->ranks, k, P[k - 1],
                                                                   xcap[k], A2);
    }
    { QTT_PROF("round_sketch", s);
    k_wl<T, R><<<GRID1((long long)lk * Rc[k])>>>(Ok, P[k - 1], P[k], A2, lk, x->ranks, k, Rc[k],
                                                 WL + wloff[k]);
    }
    { QTT_PROF("round_sketch", s);
    const unsigned nbk =
        (unsigned)std::min<long long>(device_sm_count(), ((long long)lk * Rc[k] + 255) / 256);
    k_absmax<T><<<nbk, 256, 0, s>>>(WL + wloff[k], lk, x->ranks, k, P[k], wmax + k);
    k_scale_max<T><<<nbk, 256, 0, s>>>(WL + wloff[k], lk, x->ranks, k, P[k], wmax + k);
    }
  }
  // --- 2. right-to-left orthogonalising pass
  T* Ccur = C0;
  T* Cnext = C1;
  cudaMemcpyAsync(Ccur, one, sizeof(T), cudaMemcpyDeviceToDevice, s);
  int ldc = 1;  // = Rc[d]
  for (int k = d; k >= 1; --k) {
    const R* Ok = Oc + op->off[k - 1];
    const T* Xk = Xc + x->off[k - 1];
    const int n2 = 2 * lq[k];
    { QTT_PROF("round_orth", s);
    k_b1<T><<<GRID1((long long)xcap[k - 1] * 2 * P[k] * lq[k])>>>(Xk, x->ranks, k, xcap[k - 1], P[k],
                                                                   Ccur, ldc, lq[k], d, A2);
    }
    const int ldz = Rc[k - 1];
    T* Zdst = (k == 1) ? Tpc + Tp->off[0] : Z;
    { QTT_PROF("round_orth", s);
    k_z<T, R><<<GRID1((long long)xcap[k - 1] * P[k - 1] * 2 * lq[k])>>>(Ok, P[k - 1], P[k], A2, x->ranks,
                                                                        k, xcap[k - 1], lq[k], ldz, Zdst);
    }
    if (k == 1) break;
    const int l0 = l[k - 1];
    { QTT_PROF("round_orth", s);
    k_s<T><<<GRID1((long long)l0 * n2 * KS_SPLIT)>>>(WL + wloff[k - 1], l0, Z, ldz, x->ranks, k,
                                                    P[k - 1], n2, S);
    }
    const int lq0 = lq[k - 1];
    {
      QTT_PROF("round_qr", s);
      const size_t sm = sizeof(T) * ((size_t)n2 * l0 + (size_t)n2 * lq0);
      static std::atomic<unsigned long long> qr_cfg{0};
      if (first_on_device(&qr_cfg))
        cudaFuncSetAttribute(k_house_q<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(T) * 2 * 128 * 64));
      k_house_q<T><<<1, QR_THREADS, sm, s>>>(S, l0, n2, l0, lq0, V);
    }
    const T* Vuse = V;
    { QTT_PROF("round_orth", s);
    k_qcore<T><<<GRID1(lq0 * n2)>>>(Vuse, n2, lq0, Tpc + Tp->off[k - 1]);
    }
    { QTT_PROF("round_orth", s);
    k_c<T><<<GRID1((long long)ldz * lq0)>>>(Z, ldz, Vuse, n2, lq0, x->ranks, k, P[k - 1], ldz, Cnext);
    }
    std::swap(Ccur, Cnext);
    ldc = ldz;
  }
  // Tp ranks (host-known)
  set_ranks_from_host(Tp->ranks, lq, s);
  // --- 3. left-to-right truncation
  cudaMemcpyAsync(Lc, one, sizeof(T), cudaMemcpyDeviceToDevice, s);
  T* yc = (T*)y->cores;
  for (int k = 1; k <= d; ++k) {
    const int lq0 = lq[k - 1], lqk = lq[k];
    const int tcap0 = ocap[k - 1];
    T* Ztd = (k == d) ? yc + y->off[d - 1] : Zt;
    { QTT_PROF("round_trunc", s);
    k_zt<T><<<GRID1(2 * tcap0 * lqk)>>>(Lc, y->ranks, k, tcap0, Tpc + Tp->off[k - 1], lq0, lqk, Ztd);
    }
    if (k == d) break;
    const int mcap = 2 * tcap0;
    T* corek = yc + y->off[k - 1];
    if (lqk < mcap) {
      // more rows than columns: QR first, then the rank decision on R
      {
        QTT_PROF("round_trunc_qr", s);
        static std::atomic<unsigned long long> qr_rows_cfg{0};
        if (first_on_device(&qr_rows_cfg))
          cudaFuncSetAttribute(k_qr_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(sizeof(T) * 2 * 128 * 64));
        const size_t sm = sizeof(T) * ((size_t)mcap * lqk + (size_t)mcap * lqk);
        k_qr_rows<T><<<1, QR_THREADS, sm, s>>>(Zt, y->ranks + (k - 1), 2, lqk, Qz, Rz, kd);
      }
      { QTT_PROF("round_trunc", s);
      k_gram_rows<T><<<GRID1(lqk * lqk)>>>(Rz, kd, 1, lqk, lqk, G, 128);
      }
      if (refine) {
        launch_eig_dense<T>(G, 128, kd, 1, 0, lqk, 0 /*ALL*/, eps_u, d, cap_at(k), nullptr, 0, lqk,
                            nullptr, V1, nullptr, nullptr, nullptr, y->norm2, k == 1, y->status, s);
        { QTT_PROF("round_trunc", s);
        k_proj_rows<T><<<GRID1(lqk * lqk)>>>(V1, Rz, kd, 1, nullptr, lqk, lqk, W1);
        }
        { QTT_PROF("round_trunc", s);
        k_gram_rows<T><<<GRID1(lqk * lqk)>>>(W1, kd, 1, lqk, lqk, G, 128);
        }
        launch_eig_dense<T>(G, 128, kd, 1, 0, lqk, 1 /*DECIDE*/, eps_u, d, cap_at(k), nullptr, 0,
                            lqk, V1, V, Ur, y->ranks + k, nullptr, y->norm2, 0, y->status, s, 1,
                            delta_u, -1, y->margin + k);
      } else {
        launch_eig_dense<T>(G, 128, kd, 1, 0, lqk, 1, eps_u, d, cap_at(k), nullptr, 0, lqk,
                            nullptr, Ur, nullptr, y->ranks + k, nullptr, y->norm2, k == 1,
                            y->status, s, 0, delta_u, -1, y->margin + k);
      }
      const int rcapk = ocap[k];
      { QTT_PROF("round_trunc", s);
      k_qu<T><<<GRID1(mcap * rcapk)>>>(Qz, y->ranks + (k - 1), kd, Ur, y->ranks + k, mcap, rcapk,
                                       corek);
      }
      // Lc = Ur^H R  (t_k x lq_k)
      { QTT_PROF("round_trunc", s);
      k_proj_rows<T><<<GRID1(lqk * lqk)>>>(Ur, Rz, kd, 1, y->ranks + k, lqk, lqk, Lc);
      }
      continue;
    }
    { QTT_PROF("round_trunc", s);
    k_gram_rows<T><<<GRID1(mcap * mcap)>>>(Zt, y->ranks + (k - 1), 2, mcap, lqk, G, 128);
    }
    if (refine) {
      launch_eig_dense<T>(G, 128, y->ranks + (k - 1), 2, 0, mcap, 0 /*ALL*/, eps_u, d, cap_at(k),
                          nullptr, 0, lqk, nullptr, V1, nullptr, nullptr, nullptr, y->norm2, k == 1,
                          y->status, s);
      { QTT_PROF("round_trunc", s);
      k_proj_rows<T><<<GRID1(mcap * lqk)>>>(V1, Zt, y->ranks + (k - 1), 2, nullptr, mcap, lqk, W1);
      }
      { QTT_PROF("round_trunc", s);
      k_gram_rows<T><<<GRID1(mcap * mcap)>>>(W1, y->ranks + (k - 1), 2, mcap, lqk, G, 128);
      }
      // rank decision at eps_round: small eigenvalues to relative accuracy
      launch_eig_dense<T>(G, 128, y->ranks + (k - 1), 2, 0, mcap, 1 /*DECIDE*/, eps_u, d, cap_at(k),
                          nullptr, 0, lqk, V1, V, corek, y->ranks + k, nullptr, y->norm2, 0,
                          y->status, s, 1, delta_u, -1, y->margin + k);
    } else {
      launch_eig_dense<T>(G, 128, y->ranks + (k - 1), 2, 0, mcap, 1, eps_u, d, cap_at(k), nullptr, 0,
                          lqk, nullptr, corek, nullptr, y->ranks + k, nullptr, y->norm2, k == 1,
                          y->status, s, 0, delta_u, -1, y->margin + k);
    }
    // Lc = core_k^H Zt  (t_k x lq_k)
    { QTT_PROF("round_trunc", s);
    k_proj_rows<T><<<GRID1(mcap * lqk)>>>(corek, Zt, y->ranks + (k - 1), 2, y->ranks + k, mcap, lqk,
                                          Lc);
    }
  }
  st = cuda_check(cudaGetLastError(), "round launch");
  release();
  tensor_free_async(Tp, s);
  if (st != QTT_OK) { qtt_free(y); return st; }
  *out = y;
  return QTT_OK;
}

// ---------------------------------------------------------------- large ranks
// Copy of x with every core zero-padded to the host capacities, so that the
// large-rank contractions below have host-known shapes and strides (the
// tensor is unchanged: the added bond directions carry zeros).
template <typename T>
__global__ void k_pad_core(const T* __restrict__ X, const int* __restrict__ xr, int k, int c0,
                           int c1, T* __restrict__ Xp) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)c0 * 2 * c1) return;
  const int a = (int)(e % c0);
  const long long t = e / c0;
  const int i = (int)(t % 2), b = (int)(t / 2);
  const int r0 = xr[k - 1], r1 = xr[k];
  Xp[e] = (a < r0 && b < r1) ? X[a + (size_t)r0 * (i + 2 * b)] : szero<T>();
}

// *n2 = sum |core|^2 of one core (n elements), one CTA, FP64 sum
template <typename T>
__global__ void k_core_norm2(const T* c, long long n, double* n2) {
  __shared__ double red[32];
  double a = 0.0;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) a += (double)sabs2(c[e]);
  for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *n2 = t;
  }
}
// dst keeps its own error if it has one, else takes src's
__global__ void k_status_merge(int* dst, const int* src) {
  if (threadIdx.x == 0 && *dst == 0) *dst = *src;
}

// the products of the large-rank rounding: tensor cores unless switched off
template <typename TA>
static qtt_status big_gemm(const CGemmArgs<TA>& g, int nbatch, int* status, cudaStream_t s,
                           const char* name) {
  const int mode = tc_gemm_enabled();
  const bool tc = (mode == 1) || (mode == 2 && g.K <= 64);
  return tc ? tc_cgemm<TA>(g, nbatch, status, s, name) : cgemm<TA>(g, nbatch, s, name);
}

// Rounding of Y = O X when the sketch rank exceeds QTT_RANK_CAP (complex64
// only).  Steps 1 and 2 of round_product_t -- left sketches through the
// orthonormal sketch cores, then the right-to-left randomised range finder
// per cut -- with the dense contractions as strided batched GEMMs and the
// range finder's QR by the blocked Householder QR.  The truncation sweep of
// step 3 is not run: its rank decisions would need eigen-solves beyond the
// one-CTA solvers' n <= 128, and at the accuracies this mode serves
// (eps_round ~ 1e-6, near FP32 resolution) they would keep nearly every
// sketched direction anyway.  The result is the right-orthonormal TT of
// ranks lq_k = min(sketch, 2^k, 2^(d-k), P_k r_k) (fixed-rank randomised
// rounding: its error is that of the range finder, close to the best
// approximation at ranks lq_k minus the oversampling).
static qtt_status round_product_big(const qtt_op* op, const qtt_tensor* x, int sketch,
                                    unsigned long long seed, cudaStream_t s, qtt_tensor** out) {
  using T = float2;
  using R = float;
  const int d = x->desc.d;
  if (sketch > QTT_SKETCH_CAP_BIG) {
    set_error("round: sketch rank %d above the large-rank limit %d", sketch, QTT_SKETCH_CAP_BIG);
    return QTT_EINVAL;
  }
  const std::vector<int>& P = op->P;
  const std::vector<int>& xcap = x->rcap;
  std::vector<int> Rc(d + 1), l(d + 1), lq(d + 1);
  for (int k = 0; k <= d; ++k) Rc[k] = P[k] * xcap[k];
  for (int k = 0; k <= d; ++k) {
    long long lim = std::min<long long>(1LL << std::min(k, 40), 1LL << std::min(d - k, 40));
    l[k] = (int)std::min<long long>({(long long)sketch, lim, (long long)Rc[k]});
  }
  l[0] = l[d] = 1;
  for (int k = 1; k < d; ++k) l[k] = std::min(l[k], 2 * l[k - 1]);
  lq[d] = 1;
  for (int k = d; k >= 2; --k) lq[k - 1] = std::min(l[k - 1], 2 * lq[k]);
  lq[0] = 1;
  int Rmax = 1, lmax = 1, Pmax = 1, xmax = 1;
  for (int k = 0; k <= d; ++k) {
    Rmax = std::max(Rmax, Rc[k]);
    lmax = std::max(lmax, l[k]);
    Pmax = std::max(Pmax, P[k]);
    xmax = std::max(xmax, xcap[k]);
  }
  std::vector<size_t> wloff(d), omoff(d);
  size_t wltot = 0, omtot = 0;
  for (int k = 0; k < d; ++k) { wloff[k] = wltot; wltot += (size_t)l[k] * Rc[k]; }
  for (int k = 1; k < d; ++k) { omoff[k] = omtot; omtot += (size_t)l[k - 1] * 2 * l[k]; }
  const size_t a1sz = (size_t)lmax * 2 * Rmax;
  const size_t a2sz = std::max((size_t)lmax * 2 * Pmax * 2 * xmax, (size_t)xmax * 2 * Pmax * lmax);
  T* WL = (T*)scratch_alloc(sizeof(T) * std::max<size_t>(wltot, 1), s);
  bool om_owned = false;
  R* Om = get_sketch<R>(l, omoff, omtot, d, seed, s, &om_owned);
  T* A1 = (T*)scratch_alloc(sizeof(T) * a1sz, s);
  T* A2 = (T*)scratch_alloc(sizeof(T) * a2sz, s);
  T* Z = (T*)scratch_alloc(sizeof(T) * (size_t)Rmax * 2 * lmax, s);
  T* C0 = (T*)scratch_alloc(sizeof(T) * (size_t)Rmax * lmax, s);
  T* C1 = (T*)scratch_alloc(sizeof(T) * (size_t)Rmax * lmax, s);
  T* S = (T*)scratch_alloc(sizeof(T) * (size_t)lmax * 2 * lmax, s);
  T* Aq = (T*)scratch_alloc(sizeof(T) * (size_t)lmax * 2 * lmax, s);
  T* V = (T*)scratch_alloc(sizeof(T) * (size_t)lmax * 2 * lmax, s);
  T* Tm = (T*)scratch_alloc(sizeof(T) * big_qr_tm_elems(lmax), s);
  T* one = (T*)scratch_alloc(sizeof(T), s);
  unsigned* wmax = (unsigned*)scratch_alloc(sizeof(unsigned) * (d + 1), s);
  auto release = [&]() {
    scratch_free(WL, s); if (om_owned) scratch_free(Om, s); scratch_free(A1, s); scratch_free(A2, s);
    scratch_free(Z, s); scratch_free(C0, s); scratch_free(C1, s); scratch_free(S, s);
    scratch_free(Aq, s); scratch_free(V, s); scratch_free(Tm, s); scratch_free(one, s);
    scratch_free(wmax, s);
  };
  if (!WL || !Om || !A1 || !A2 || !Z || !C0 || !C1 || !S || !Aq || !V || !Tm || !one || !wmax) {
    release();
    if (!Om && WL && A1) set_error("round: sketch generation failed");
    else set_error("round: large-rank scratch allocation failed");
    return QTT_ENOMEM;
  }
  k_one<<<1, 32, 0, s>>>(one, 0);
  cudaMemsetAsync(wmax, 0, sizeof(unsigned) * (d + 1), s);
  // x padded to its capacities
  qtt_tensor* xp = nullptr;
  qtt_status st = tensor_alloc(x->desc, xcap, s, &xp);
  if (st != QTT_OK) { release(); return st; }
  for (int k = 1; k <= d; ++k) {
    const long long n = (long long)xcap[k - 1] * 2 * xcap[k];
    QTT_PROF("round_pad", s);
    k_pad_core<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const T*)x->cores + x->off[k - 1],
                                                             x->ranks, k, xcap[k - 1], xcap[k],
                                                             (T*)xp->cores + xp->off[k - 1]);
  }
  set_ranks_from_host(xp->ranks, xcap, s);
  // output: the right-orthonormal TT of ranks lq
  qtt_tensor* y = nullptr;
  st = tensor_alloc(x->desc, lq, s, &y);
  if (st != QTT_OK) { tensor_free_async(xp, s); release(); return st; }
  const R* Oc = (const R*)op->cores;
  const T* Xc = (const T*)xp->cores;
  T* yc = (T*)y->cores;

  // --- 1. left sketches
  cudaMemcpyAsync(WL + wloff[0], one, sizeof(T), cudaMemcpyDeviceToDevice, s);
  for (int k = 1; k < d && st == QTT_OK; ++k) {
    const int l0 = l[k - 1], lk = l[k];
    const int r0 = xcap[k - 1], r1 = xcap[k];
    const int Pin = P[k - 1];
    const R* Ok = Oc + op->off[k - 1];
    const T* Xk = Xc + xp->off[k - 1];
    {  // A1[s + lk (j + 2 c)] = sum_{s'} Om[s' + l0 (j + 2 s)] WL0[s' + l0 c]
      CGemmArgs<R> g;
      g.A = Om + omoff[k]; g.sAi = 2LL * l0; g.sAk = 1; g.bA1 = l0;
      g.B = WL + wloff[k - 1]; g.sBk = 1; g.sBj = l0;
      g.C = A1; g.sCi = 1; g.sCj = 2LL * lk; g.bC1 = lk;
      g.M = lk; g.N = Rc[k - 1]; g.K = l0; g.nb1 = 2;
      st = big_gemm<R>(g, 2, y->status, s, "gemm_sketch_a1");
    }
    if (st != QTT_OK) break;
    {  // A2[rho + 2lk (p + Pin (i + 2 b))] = sum_a A1[rho + 2lk (a + r0 p)] X[a + r0 (i + 2 b)]
      CGemmArgs<T> g;
      g.A = A1; g.sAi = 1; g.sAk = 2LL * lk; g.bA1 = 2LL * lk * r0;
      g.B = Xk; g.sBk = 1; g.sBj = r0;
      g.C = A2; g.sCi = 1; g.sCj = 2LL * lk * Pin; g.bC1 = 2LL * lk;
      g.M = 2 * lk; g.N = 2 * r1; g.K = r0; g.nb1 = Pin;
      st = big_gemm<T>(g, Pin, y->status, s, "gemm_sketch_a2");
    }
    if (st != QTT_OK) break;
    { QTT_PROF("round_sketch", s);
    k_wl<T, R><<<GRID1((long long)lk * Rc[k])>>>(Ok, Pin, P[k], A2, lk, xp->ranks, k, Rc[k],
                                                 WL + wloff[k]);
    }
    { QTT_PROF("round_sketch", s);
    const unsigned nbk = (unsigned)std::min<long long>(1024, ((long long)lk * Rc[k] + 255) / 256);
    k_absmax<T><<<nbk, 256, 0, s>>>(WL + wloff[k], lk, xp->ranks, k, P[k], wmax + k);
    k_scale_max<T><<<nbk, 256, 0, s>>>(WL + wloff[k], lk, xp->ranks, k, P[k], wmax + k);
    }
  }
  // --- 2. right-to-left range finder
  T* Ccur = C0;
  T* Cnext = C1;
  if (st == QTT_OK) cudaMemcpyAsync(Ccur, one, sizeof(T), cudaMemcpyDeviceToDevice, s);
  int ldc = 1;
  for (int k = d; k >= 1 && st == QTT_OK; --k) {
    const R* Ok = Oc + op->off[k - 1];
    const T* Xk = Xc + xp->off[k - 1];
    const int r0 = xcap[k - 1], r1 = xcap[k];
    const int Pin = P[k - 1], Pout = P[k];
    const int n2 = 2 * lq[k];
    {  // B1[a + r0 (i + 2 (q + Pout t))] = sum_b X[a + r0 (i + 2 b)] C[(b + r1 q) + ldc t]
      CGemmArgs<T> g;
      g.A = Xk; g.sAi = 1; g.sAk = 2LL * r0; g.bA1 = r0;
      g.B = Ccur; g.sBk = 1; g.sBj = ldc; g.bB2 = r1;
      g.C = A2; g.sCi = 1; g.sCj = 2LL * r0 * Pout; g.bC1 = r0; g.bC2 = 2LL * r0;
      g.M = r0; g.N = lq[k]; g.K = r1; g.nb1 = 2;
      st = big_gemm<T>(g, 2 * Pout, y->status, s, "gemm_orth_b1");
    }
    if (st != QTT_OK) break;
    const int ldz = Rc[k - 1];
    T* Zdst = (k == 1) ? yc + y->off[0] : Z;
    { QTT_PROF("round_orth", s);
    k_z<T, R><<<GRID1((long long)r0 * Pin * 2 * lq[k])>>>(Ok, Pin, Pout, A2, xp->ranks, k, r0,
                                                          lq[k], ldz, Zdst);
    }
    if (k == 1) break;
    const int l0 = l[k - 1], lq0 = lq[k - 1];
    {  // S = WL_{k-1} Z  (l0 x n2)
      CGemmArgs<T> g;
      g.A = WL + wloff[k - 1]; g.sAi = 1; g.sAk = l0;
      g.B = Z; g.sBk = 1; g.sBj = ldz;
      g.C = S; g.sCi = 1; g.sCj = l0;
      g.M = l0; g.N = n2; g.K = ldz;
      st = big_gemm<T>(g, 1, y->status, s, "gemm_orth_s");
    }
    if (st != QTT_OK) break;
    if (n2 <= QR_MAXM && l0 <= 64 && lq0 <= 64) {
      // small cut: the one-CTA Householder QR of the rank-64 path (one launch)
      QTT_PROF("round_qr", s);
      static std::atomic<unsigned long long> qr_cfg_big{0};
      if (first_on_device(&qr_cfg_big))
        cudaFuncSetAttribute(k_house_q<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(T) * 2 * 128 * 64));
      const size_t sm = sizeof(T) * ((size_t)n2 * l0 + (size_t)n2 * lq0);
      k_house_q<T><<<1, QR_THREADS, sm, s>>>(S, l0, n2, l0, lq0, V);
    } else {
      { QTT_PROF("round_qr", s);
      launch_conj_transpose<T>(S, l0, l0, n2, Aq, s);
      }
      st = big_qr_q<T>(Aq, n2, l0, lq0, V, Tm, s);
      if (st != QTT_OK) break;
    }
    { QTT_PROF("round_orth", s);
    k_qcore<T><<<GRID1(lq0 * n2)>>>(V, n2, lq0, yc + y->off[k - 1]);
    }
    {  // Cn = Z V  (ldz x lq0)
      CGemmArgs<T> g;
      g.A = Z; g.sAi = 1; g.sAk = ldz;
      g.B = V; g.sBk = 1; g.sBj = n2;
      g.C = Cnext; g.sCi = 1; g.sCj = ldz;
      g.M = ldz; g.N = lq0; g.K = n2;
      st = big_gemm<T>(g, 1, y->status, s, "gemm_orth_c");
    }
    std::swap(Ccur, Cnext);
    ldc = ldz;
  }
  if (st == QTT_OK) {
    set_ranks_from_host(y->ranks, lq, s);
    // the cores after the first are right-orthonormal: ||y||^2 = ||core_1||^2
    k_core_norm2<T><<<1, 256, 0, s>>>(yc + y->off[0], (long long)2 * lq[1], y->norm2);
    k_status_merge<<<1, 32, 0, s>>>(y->status, x->status);
    st = cuda_check(cudaGetLastError(), "round (large ranks) launch");
  }
  release();
  tensor_free_async(xp, s);
  if (st != QTT_OK) { qtt_free(y); return st; }
  *out = y;
  return QTT_OK;
}

qtt_status round_product(const qtt_op* op, const qtt_tensor* x, const qtt_trunc& tr, int sketch,
                         unsigned long long seed, cudaStream_t s, qtt_tensor** out) {
  if (op->d != x->desc.d) { set_error("round: operator/tensor mode count mismatch"); return QTT_EINVAL; }
  if (op->dt != x->desc.dt) { set_error("round: operator/tensor dtype mismatch"); return QTT_EINVAL; }
  if (op->cplx) { set_error("round: complex operators are applied by matvec"); return QTT_EUNSUPPORTED; }
  if (sketch > QTT_RANK_CAP) {
    if (x->desc.dt != QTT_C64) {
      set_error("round: sketch ranks above %d need complex64 data", QTT_RANK_CAP);
      return QTT_EUNSUPPORTED;
    }
    return round_product_big(op, x, sketch, seed, s, out);
  }
  if (x->desc.dt == QTT_F64) return round_product_t<double>(op, x, tr, sketch, seed, s, out);
  return round_product_t<float2>(op, x, tr, sketch, seed, s, out);
}

}  // namespace qtt
