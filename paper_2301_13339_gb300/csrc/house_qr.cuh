// One-CTA Householder QR building blocks (QR_THREADS threads, at most
// QR_MAXM rows), shared by the
// rounding's orthogonalisation (k_round.cu) and the TT-SVD levels that keep
// full rank (k_svd.cu).  LAPACK's convention: H_k = I - tau_k v_k v_k^H,
// v_k = [1; A[k+1:, k]], Q = H_1 ... H_kmax; the trailing matrix is updated
// with H_k^H, so the upper triangle of A ends as R with A = Q R.
#pragma once
#include "qtt_internal.cuh"

namespace qtt {

constexpr int QR_THREADS = 512;
constexpr int QR_MAXM = 128;   // rows held 4 per lane

// Reflector k from column k of A (rows k..m-1) by one warp, in the data's
// precision, on the column scaled by its largest entry (no underflow or
// overflow of |alpha - beta|^2 whatever the data's scale; tau and v are
// scale free).  Writes v below the diagonal, beta on it and tau_k.
template <typename T>
__device__ void house_form_reflector(T* A, int m, int k, T* s_tau) {
  using R = typename Sc<T>::R;
  const int lane = threadIdx.x & 31;
  R amax = (R)0;
  for (int i = k + lane; i < m; i += 32) {
    const T x = A[i + (size_t)m * k];
    amax = rmax(amax, rmax(rabs(sreal(x)), rabs(simag(x))));
  }
  for (int off = 16; off > 0; off >>= 1) amax = rmax(amax, __shfl_xor_sync(0xffffffffu, amax, off));
  T tau = szero<T>(), scal = szero<T>();
  if (amax > (R)0) {
    const R inv = (R)1 / amax;
    R part = (R)0;
    for (int i = k + 1 + lane; i < m; i += 32) part += sabs2(rscale(A[i + (size_t)m * k], inv));
    part = warp_sum(part);
    const T al = rscale(A[k + (size_t)m * k], inv);
    const R ax = sreal(al), ay = simag(al);
    if (part > (R)0 || ay != (R)0) {
      const R nrm = sqrt(ax * ax + ay * ay + part);
      const R beta = (ax >= (R)0) ? -nrm : nrm;
      const R rb = (R)1 / beta;
      tau = make_scalar<T>((beta - ax) * rb, -ay * rb);
      const R dr = ax - beta, di = ay, rden = (R)1 / (dr * dr + di * di);
      scal = rscale(make_scalar<T>(dr * rden, -di * rden), inv);   // 1 / (alpha - beta)
      for (int i = k + 1 + lane; i < m; i += 32)
        A[i + (size_t)m * k] = smul(A[i + (size_t)m * k], scal);
      if (lane == 0) A[k + (size_t)m * k] = make_scalar<T>(beta * amax, (R)0);
    }
  }
  if (lane == 0) s_tau[k] = tau;
}

// v_k = [0 (rows < k); 1; A[k+1:, k]] in registers, rows lane + 32 x
template <typename T>
__device__ __forceinline__ void house_load_v(const T* A, int m, int k, T (&v)[4]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int i = lane + 32 * x;
    v[x] = (i == k) ? sone(T()) : (i > k && i < m) ? A[i + (size_t)m * k] : szero<T>();
  }
}

// X[:, j0] and X[:, j1] <- (I - t v v^H) X[:, j] (ld m); j1 < 0: j0 only.
// One warp; the two reductions are interleaved.
template <typename T>
__device__ __forceinline__ void house_apply2(T* X, int m, const T (&v)[4], T t, int j0, int j1) {
  const int lane = threadIdx.x & 31;
  T x0[4], x1[4];
  T w0 = szero<T>(), w1 = szero<T>();
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int i = lane + 32 * x;
    x0[x] = (i < m) ? X[i + (size_t)m * j0] : szero<T>();
    x1[x] = (j1 >= 0 && i < m) ? X[i + (size_t)m * j1] : szero<T>();
    macc(w0, v[x], x0[x]);
    macc(w1, v[x], x1[x]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    w0 = sadd(w0, shfl_xor_s(w0, off));
    w1 = sadd(w1, shfl_xor_s(w1, off));
  }
  const T f0 = smul(t, w0), f1 = smul(t, w1);
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int i = lane + 32 * x;
    if (i < m) {
      X[i + (size_t)m * j0] = ssub(x0[x], smul(v[x], f0));
      if (j1 >= 0) X[i + (size_t)m * j1] = ssub(x1[x], smul(v[x], f1));
    }
  }
}

// In place on A (m x nc, ld m, shared memory, m <= QR_MAXM): R in the upper
// triangle, the v_k below the diagonal, tau_k in s_tau (shared,
// >= min(m, nc)).  One barrier per reflector: warp 0 updates column k+1
// first and forms reflector k+1 from it (look-ahead) while the other warps
// update the remaining trailing columns with reflector k.
template <typename T>
__device__ void house_qr_factor(T* A, int m, int nc, T* s_tau) {
  const int warp = threadIdx.x >> 5, nw = QR_THREADS / 32;
  const int kmax = min(m, nc);
  if (kmax > 0 && warp == 0) house_form_reflector(A, m, 0, s_tau);
  __syncthreads();
  for (int k = 0; k < kmax; ++k) {
    // trailing columns: A <- (I - conj(tau) v v^H) A
    const T ctau = conjg(s_tau[k]);
    T v[4];
    house_load_v(A, m, k, v);
    if (warp == 0) {
      if (k + 1 < nc) {
        house_apply2(A, m, v, ctau, k + 1, -1);
        __syncwarp();
        if (k + 1 < kmax) house_form_reflector(A, m, k + 1, s_tau);
      }
    } else {
      for (int j = k + 2 + (warp - 1); j < nc; j += 2 * (nw - 1)) {
        const int j1 = j + (nw - 1);
        house_apply2(A, m, v, ctau, j, j1 < nc ? j1 : -1);
      }
    }
    __syncthreads();
  }
}

// E (m x nq, ld m, shared) = the first nq columns of H_1 ... H_kmax.  H_k
// leaves e_j (j < k) unchanged, so step k touches columns j >= k only.
template <typename T>
__device__ void house_form_q(const T* A, int m, int kmax, int nq, const T* s_tau, T* E) {
  const int tid = threadIdx.x, warp = tid >> 5, nw = QR_THREADS / 32;
  for (int e = tid; e < m * nq; e += QR_THREADS) {
    const int i = e % m, j = e / m;
    E[e] = (i == j) ? sone(T()) : szero<T>();
  }
  __syncthreads();
  for (int k = kmax - 1; k >= 0; --k) {
    const T tau = s_tau[k];
    T v[4];
    house_load_v(A, m, k, v);
    for (int j = k + warp; j < nq; j += 2 * nw) {
      const int j1 = j + nw;
      house_apply2(E, m, v, tau, j, j1 < nq ? j1 : -1);
    }
    __syncthreads();
  }
}

}  // namespace qtt
