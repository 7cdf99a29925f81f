// One-CTA Householder QR building blocks (QR_THREADS threads), shared by the
// rounding's orthogonalisation (k_round.cu) and the TT-SVD levels that keep
// full rank (k_svd.cu).  LAPACK's convention: H_k = I - tau_k v_k v_k^H,
// v_k = [1; A[k+1:, k]], Q = H_1 ... H_kmax; the trailing matrix is updated
// with H_k^H, so the upper triangle of A ends as R with A = Q R.
#pragma once
#include "qtt_internal.cuh"

namespace qtt {

constexpr int QR_THREADS = 256;

// In place on A (m x nc, ld m, shared memory): R in the upper triangle,
// the v_k below the diagonal, tau_k in s_tau (shared, >= min(m, nc)).
template <typename T>
__device__ void house_qr_factor(T* A, int m, int nc, T* s_tau) {
  using R = typename Sc<T>::R;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = QR_THREADS / 32;
  const int kmax = min(m, nc);
  for (int k = 0; k < kmax; ++k) {
    // warp 0 forms the reflector and v in the data's precision, on the
    // column scaled by its largest entry (no underflow or overflow of
    // |alpha - beta|^2 whatever the data's scale; tau and v are scale free)
    if (warp == 0) {
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
    __syncthreads();
    const T tau = s_tau[k];
    // trailing columns: A <- (I - conj(tau) v v^H) A, v = [1; A[k+1:, k]]
    const T ctau = conjg(tau);
    for (int j = k + 1 + warp; j < nc; j += nw) {
      T w = szero<T>();
      for (int i = k + lane; i < m; i += 32) {
        const T vi = (i == k) ? sone(T()) : A[i + (size_t)m * k];
        macc(w, vi, A[i + (size_t)m * j]);
      }
      w = warp_sum(w);
      const T f = smul(ctau, w);
      for (int i = k + lane; i < m; i += 32) {
        const T vi = (i == k) ? sone(T()) : A[i + (size_t)m * k];
        A[i + (size_t)m * j] = ssub(A[i + (size_t)m * j], smul(vi, f));
      }
    }
    __syncthreads();
  }
}

// E (m x nq, ld m, shared) = the first nq columns of H_1 ... H_kmax.
template <typename T>
__device__ void house_form_q(const T* A, int m, int kmax, int nq, const T* s_tau, T* E) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = QR_THREADS / 32;
  // Q = H_1 ... H_kmax applied to the first nq columns of I
  for (int e = tid; e < m * nq; e += QR_THREADS) {
    const int i = e % m, j = e / m;
    E[e] = (i == j) ? sone(T()) : szero<T>();
  }
  __syncthreads();
  for (int k = kmax - 1; k >= 0; --k) {
    const T tau = s_tau[k];
    for (int j = warp; j < nq; j += nw) {
      T w = szero<T>();
      for (int i = k + lane; i < m; i += 32) {
        const T vi = (i == k) ? sone(T()) : A[i + (size_t)m * k];
        macc(w, vi, E[i + (size_t)m * j]);
      }
      w = warp_sum(w);
      const T f = smul(tau, w);
      for (int i = k + lane; i < m; i += 32) {
        const T vi = (i == k) ? sone(T()) : A[i + (size_t)m * k];
        E[i + (size_t)m * j] = ssub(E[i + (size_t)m * j], smul(vi, f));
      }
    }
    __syncthreads();
  }
}

}  // namespace qtt
