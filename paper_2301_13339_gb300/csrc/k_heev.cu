// Hermitian eigensolver for the FP32 path (complex float, n <= 128).
//
// The Gram matrices of the TT-SVD steps (Alg. 1) and of the rounding sweep
// are factored as G = U L U^H by
//   1. Householder reduction to a real symmetric tridiagonal T = Q^H G Q
//      (n-1 reflectors H_k = I - tau_k v_k v_k^H, LAPACK's convention);
//   2. all eigenvalues of T by bisection on Sturm counts, 4 threads per
//      eigenvalue evaluating 4 interior points (5-section) per round;
//   3. eigenvectors of T for the wanted eigenvalues by the twisted
//      factorisation T - lambda I = N_k D_k N_k^T (one thread per vector);
//   4. modified Gram-Schmidt, twice, inside clusters of close eigenvalues;
//   5. Newton-Schulz steps and U = Q Z.
// Steps 1-4 run in one CTA (heev_tri_kernel).  For n <= 32 the same kernel
// does step 5 too (8 threads per column of U); above, it hands Z and the
// reflectors to heev_back_kernel, a cluster of 8 CTAs that splits the
// columns (distributed shared memory for the Newton-Schulz exchange, 16
// threads per column for the back-transformation).  About 10-20x fewer
// dependent steps than cyclic Jacobi (n-1 steps per sweep, ~8 sweeps).  Same
// EigArgs contract as the Jacobi kernels in k_svd.cu.
#include "qtt_internal.cuh"
#include <cooperative_groups.h>
#include <algorithm>
#include <cfloat>

namespace qtt {

constexpr int HT = 512;
constexpr int HMAX = 128;

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconjf(float2 a) { return make_float2(a.x, -a.y); }

// Twisted factorisation eigenvector of the tridiagonal (d, e) for sigma,
// written to z[0..n).  Scratch um[] holds U- (local memory).
__device__ void twisted_vector(const float* d, const float* e, int n, float sigma, float pivmin,
                               float* z) {
  float um[HMAX];
  // stationary (top-down): L+_i, stored in z[i]
  float D = d[0] - sigma;
  for (int i = 0; i < n - 1; ++i) {
    if (fabsf(D) < pivmin) D = -pivmin;
    const float l = e[i] / D;
    z[i] = l;
    D = d[i + 1] - sigma - l * e[i];
  }
  // progressive (bottom-up): U-_i
  D = d[n - 1] - sigma;
  for (int i = n - 2; i >= 0; --i) {
    if (fabsf(D) < pivmin) D = pivmin;
    const float u = e[i] / D;
    um[i] = u;
    D = d[i] - sigma - u * e[i];
  }
  // twist index: minimal |gamma_k|
  int kbest = 0;
  float gbest = FLT_MAX;
  for (int k = 0; k < n; ++k) {
    float g = d[k] - sigma;
    if (k > 0) g -= z[k - 1] * e[k - 1];
    if (k < n - 1) g -= um[k] * e[k];
    if (fabsf(g) < gbest) { gbest = fabsf(g); kbest = k; }
  }
  const int k = kbest;
  // z_k = 1; z_i = -L+_i z_{i+1} (i < k); z_{i+1} = -U-_i z_i (i >= k)
  float zn = 1.f;
  float prev = 1.f;
  for (int i = k - 1; i >= 0; --i) {
    const float v = -z[i] * prev;
    z[i] = v;
    prev = v;
  }
  z[k] = 1.f;
  prev = 1.f;
  for (int i = k; i < n - 1; ++i) {
    const float v = -um[i] * prev;
    z[i + 1] = v;
    prev = v;
  }
  // normalise with a scaling by the largest entry (the recurrences can
  // reach ~1/pivmin next to a tiny pivot); an overflow falls back to e_k,
  // which the orthogonalisation step then treats as a degenerate copy
  float zmax = 0.f;
  bool finite = true;
  for (int i = 0; i < n; ++i) {
    finite = finite && isfinite(z[i]);
    zmax = fmaxf(zmax, fabsf(z[i]));
  }
  if (!finite || !(zmax > 0.f)) {
    for (int i = 0; i < n; ++i) z[i] = (i == k) ? 1.f : 0.f;
    return;
  }
  const float inv = 1.f / zmax;
  float s2 = 0.f;
  for (int i = 0; i < n; ++i) {
    const float t = z[i] * inv;
    s2 = fmaf(t, t, s2);
  }
  zn = inv * rsqrtf(s2);
  for (int i = 0; i < n; ++i) z[i] *= zn;
}

// Number of eigenvalues of the tridiagonal (d, e2 = e^2) smaller than x.
__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int n, float x,
                                           float pivmin) {
  int c = 0;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  c += (q < 0.f);
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += (q < 0.f);
  }
  return c;
}

// Hand-off of a split solve: the tridiagonal eigenvectors Z (n x ncopy, ld n),
// the packed reflectors (reflector k, rows k+2..n-1, at sum_{k'<k}(n-k'-2)),
// tau, and hdr[0] = ncopy.  Z == nullptr: one kernel does everything.
struct HeevSplit {
  float* Z;
  float2* V;
  float2* tau;
  int* hdr;
};

__global__ void __launch_bounds__(HT) heev_tri_kernel(EigArgs<float2> a, HeevSplit hs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float s_d[HMAX], s_e[HMAX], s_e2[HMAX], s_lam[HMAX];
  __shared__ float2 s_tau[HMAX], s_v[HMAX], s_p[HMAX];
  __shared__ float s_redf[HT / 32];
  __shared__ float s_red4[4];
  __shared__ float2 s_pdw[HT / 32];
  __shared__ double s_redd[HT / 32];
  __shared__ float s_xn2, s_glo, s_ghi, s_pivmin;
  __shared__ double s_trace;
  __shared__ int s_r, s_clu[HMAX], s_pack[HT / 32];
  __shared__ float2 s_part[4][HMAX];
  __shared__ int s_bad[HMAX], s_cend[HMAX];
  __shared__ float s_inv[HMAX];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.mg_ptr ? a.mg_mul * (*a.mg_ptr) : a.mg_const;
#ifdef QTT_HEEV_TRI_PROFILE
#define HEEV_STAMP(i) \
  do { if (a.phase_clk && tid == 0 && (i) < 6) a.phase_clk[i] = clock64(); } while (0)
#else
#define HEEV_STAMP(i) \
  do { if (a.phase_clk && tid == 0) a.phase_clk[i] = clock64(); } while (0)
#endif
  HEEV_STAMP(0);
  float2* A = reinterpret_cast<float2*>(smem_raw);        // n x n, ld n
  float* Z = reinterpret_cast<float*>(A + (size_t)n * n);  // n x n, ld ldz = n + 1
  const int ldz = n + 1;

  // ---- trace, then the Gram (double) scaled to unit trace in FP32: the
  // solver works on O(1) numbers whatever the data's scale (no overflow or
  // underflow in the reflectors); eigenvalues are scaled back by the trace
  double trl = 0.0;
  for (int i = tid; i < n; i += HT) trl += a.G[i + (size_t)a.ldp * i].x;
  for (int off = 16; off > 0; off >>= 1) trl += __shfl_xor_sync(0xffffffffu, trl, off);
  if (lane == 0) s_redd[warp] = trl;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < HT / 32; ++w) t += s_redd[w];
    if (a.write_norm2) *a.norm2 = t;
    s_trace = (t > 0.0 && isfinite(t)) ? t : 1.0;
  }
  __syncthreads();
  const double gsc = 1.0 / s_trace;
  for (int e = tid; e < n * n; e += HT) {
    const int i = e % n, j = e / n;
    double2 g = a.G[i + (size_t)a.ldp * j];
    if (i == j) g.y = 0.0;
    A[e] = make_float2((float)(g.x * gsc), (float)(g.y * gsc));
  }
  __syncthreads();

  HEEV_STAMP(1);
  // ---- 1. Householder tridiagonalisation (lower).  Per column k, all
  // phases spread over the block (5 barriers): the column norm by the 128
  // row threads; the reflector scalars computed redundantly by every thread
  // (no serial section) and v formed by the row threads; the partial
  // products of A22 v together with the partial sums of (A22 v)^H v (p^H v
  // is linear in them); w = p + alpha2 v by the row threads; the rank-2
  // update A22 -= v w^H + w v^H.
#ifdef QTT_HEEV_TRI_PROFILE
  long long tp_acc[4] = {0, 0, 0, 0}, tp_t = clock64();
#define TRI_MARK(i) do { if (tid == 0) { const long long t_ = clock64(); tp_acc[i] += t_ - tp_t; tp_t = t_; } } while (0)
#else
#define TRI_MARK(i) do { } while (0)
#endif
  for (int k = 0; k < n - 1; ++k) {
    const int irow = k + 1 + tid;                 // row of the threads tid < 128
    const bool rowt = (tid < 128) && (irow < n);
    float2 xk = make_float2(0.f, 0.f);
    if (tid < 128) {
      float part = 0.f;
      if (rowt) {
        xk = A[irow + (size_t)n * k];
        if (irow >= k + 2) part = fmaf(xk.x, xk.x, xk.y * xk.y);
      }
      part = warp_sum(part);
      if (lane == 0) s_red4[warp] = part;
    }
    __syncthreads();
    // on the unit-trace matrix a column below 1e-18 is negligible (and
    // would underflow |alpha - beta|^2): it is left as it is
    const float xn2 = (s_red4[0] + s_red4[1]) + (s_red4[2] + s_red4[3]);
    const float2 al = A[(k + 1) + (size_t)n * k];
    float2 tau = make_float2(0.f, 0.f), scal = make_float2(0.f, 0.f);
    float beta = al.x;
    const float nrm = sqrtf(al.x * al.x + al.y * al.y + xn2);
    if ((xn2 > 0.f || al.y != 0.f) && nrm > 1e-18f) {
      beta = (al.x >= 0.f) ? -nrm : nrm;
      const float rb = 1.f / beta;
      tau = make_float2((beta - al.x) * rb, -al.y * rb);
      const float dr = al.x - beta, di = al.y, rden = 1.f / (dr * dr + di * di);
      scal = make_float2(dr * rden, -di * rden);
    }
    const bool act = (tau.x != 0.f || tau.y != 0.f);   // identical in every thread
    if (rowt) {
      float2 v = make_float2(1.f, 0.f);
      if (irow > k + 1) {
        v = act ? cmulf(xk, scal) : xk;
        if (act) A[irow + (size_t)n * k] = v;
      }
      s_v[irow] = v;
    }
    if (tid == 0) {
      s_e[k] = beta;
      s_d[k] = A[k + (size_t)n * k].x;
      s_tau[k] = tau;
    }
    __syncthreads();
    TRI_MARK(0);
    if (!act) continue;   // uniform; the barrier above ends every read of s_red4
    // partial products of A22 v: thread t owns row k+1+(t & 127) and the
    // columns congruent to (t >> 7) mod 4; lanes of a warp read consecutive rows
    {
      const int i = k + 1 + (tid & 127), ph = tid >> 7;
      float2 acc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = make_float2(0.f, 0.f);
      float2 vi = make_float2(0.f, 0.f);
      if (i < n) {
        vi = s_v[i];
        int j = k + 1 + ph;
        // four independent chains (columns j, j+4, j+8, j+12)
        for (; j + 12 < n; j += 16) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 aij = A[i + (size_t)n * (j + 4 * u)], vj = s_v[j + 4 * u];
            acc[u].x = fmaf(aij.x, vj.x, fmaf(-aij.y, vj.y, acc[u].x));
            acc[u].y = fmaf(aij.x, vj.y, fmaf(aij.y, vj.x, acc[u].y));
          }
        }
        for (; j < n; j += 4) {
          const float2 aij = A[i + (size_t)n * j], vj = s_v[j];
          acc[0].x = fmaf(aij.x, vj.x, fmaf(-aij.y, vj.y, acc[0].x));
          acc[0].y = fmaf(aij.x, vj.y, fmaf(aij.y, vj.x, acc[0].y));
        }
      }
      const float2 a4 = make_float2(acc[0].x + acc[1].x + acc[2].x + acc[3].x,
                                    acc[0].y + acc[1].y + acc[2].y + acc[3].y);
      s_part[ph][tid & 127] = a4;
      // conj(a4) v_i, summed over the block = (A22 v)^H v
      float2 pd = make_float2(fmaf(a4.x, vi.x, a4.y * vi.y), fmaf(a4.x, vi.y, -a4.y * vi.x));
      pd = warp_sum(pd);
      if (lane == 0) s_pdw[warp] = pd;
    }
    __syncthreads();
    TRI_MARK(1);
    if (rowt) {
      // p = tau A22 v; p^H v = conj(tau) (A22 v)^H v; w = p + alpha2 v with
      // alpha2 = -tau (p^H v) / 2
      const int il = irow - k - 1;
      float2 acc = s_part[0][il];
      for (int ph = 1; ph < 4; ++ph) { acc.x += s_part[ph][il].x; acc.y += s_part[ph][il].y; }
      float2 sv = make_float2(0.f, 0.f);
      for (int w = 0; w < HT / 32; ++w) { sv.x += s_pdw[w].x; sv.y += s_pdw[w].y; }
      const float2 pdt = cmulf(cconjf(tau), sv);
      const float2 t2 = cmulf(tau, pdt);
      const float2 al2 = make_float2(-0.5f * t2.x, -0.5f * t2.y);
      const float2 pi = cmulf(tau, acc), vi = s_v[irow];
      float2 w = pi;
      w.x = fmaf(al2.x, vi.x, fmaf(-al2.y, vi.y, w.x));
      w.y = fmaf(al2.x, vi.y, fmaf(al2.y, vi.x, w.y));
      s_p[irow] = w;
    }
    __syncthreads();
    TRI_MARK(2);
    // A22 -= v w^H + w v^H: thread t owns row k+1+(t & 127), columns in
    // steps of 4 from k+1+(t >> 7)
    {
      const int i = k + 1 + (tid & 127);
      if (i < n) {
        const float2 vi = s_v[i], wi = s_p[i];
#pragma unroll 4
        for (int j = k + 1 + (tid >> 7); j < n; j += 4) {
          const float2 vj = s_v[j], wj = s_p[j];
          float2 x = A[i + (size_t)n * j];
          // x -= vi conj(wj) + wi conj(vj)
          x.x -= vi.x * wj.x + vi.y * wj.y + wi.x * vj.x + wi.y * vj.y;
          x.y -= vi.y * wj.x - vi.x * wj.y + wi.y * vj.x - wi.x * vj.y;
          A[i + (size_t)n * j] = x;
        }
      }
    }
    __syncthreads();
    TRI_MARK(3);
  }
#ifdef QTT_HEEV_TRI_PROFILE
  // diagnostic build only: the four sub-phase totals of the reduction
  if (tid == 0 && a.phase_clk) for (int i = 0; i < 4; ++i) a.phase_clk[6 + i] = tp_acc[i];
#endif
#undef TRI_MARK
  if (tid == 0) {
    s_d[n - 1] = A[(n - 1) + (size_t)n * (n - 1)].x;
    float glo = FLT_MAX, ghi = -FLT_MAX, me2 = 0.f;
    for (int i = 0; i < n; ++i) {
      const float r = (i > 0 ? fabsf(s_e[i - 1]) : 0.f) + (i < n - 1 ? fabsf(s_e[i]) : 0.f);
      glo = fminf(glo, s_d[i] - r);
      ghi = fmaxf(ghi, s_d[i] + r);
      if (i < n - 1) {
        s_e2[i] = s_e[i] * s_e[i];
        me2 = fmaxf(me2, s_e2[i]);
      }
    }
    const float tn = fmaxf(fabsf(glo), fabsf(ghi));
    s_pivmin = FLT_MIN * fmaxf(1.f, me2);
    s_glo = glo - 4.f * FLT_EPSILON * tn - 2.f * s_pivmin;
    s_ghi = ghi + 4.f * FLT_EPSILON * tn + 2.f * s_pivmin;
  }
  __syncthreads();

  HEEV_STAMP(2);
  // ---- 2. eigenvalues: 5-section with 4 threads per eigenvalue (ascending index)
  {
    const int g = tid >> 2, sub = tid & 3;
    const float pivmin = s_pivmin;
    for (int base = 0; base < n; base += HT / 4) {
      const int idx = base + g;                 // all 4 lanes of a group share idx
      float lo = s_glo, hi = s_ghi;
      const bool act = idx < n;
      for (int it = 0; it < 48; ++it) {
        const float w = hi - lo;
        const bool done = !(w > 2.f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi)) + 4.f * pivmin);
        // the 4 lanes of a group agree on done; groups converge independently
        const unsigned ballot = __ballot_sync(0xffffffffu, act && !done);
        if (ballot == 0u) break;
        const float x = lo + w * (float)(sub + 1) * 0.2f;
        const int c = (act && !done) ? sturm_count(s_d, s_e2, n, x, pivmin) : 0;
        // gather the 4 counts of the group
        const int gl = lane & ~3;
        const int c0 = __shfl_sync(0xffffffffu, c, gl + 0);
        const int c1 = __shfl_sync(0xffffffffu, c, gl + 1);
        const int c2 = __shfl_sync(0xffffffffu, c, gl + 2);
        const int c3 = __shfl_sync(0xffffffffu, c, gl + 3);
        if (act && !done) {
          const float x0 = lo + w * 0.2f, x1 = lo + w * 0.4f, x2 = lo + w * 0.6f, x3 = lo + w * 0.8f;
          if (c0 > idx) hi = x0;
          else if (c1 > idx) { lo = x0; hi = x1; }
          else if (c2 > idx) { lo = x1; hi = x2; }
          else if (c3 > idx) { lo = x2; hi = x3; }
          else lo = x3;
        }
      }
      if (act && sub == 0) {
        const float lam = 0.5f * (lo + hi);
        if (!isfinite(lam) && a.status) atomicOr(a.status, DEV_ST_NONFINITE);
        s_lam[idx] = lam;
      }
    }
  }
  __syncthreads();

  // ---- rank decision on the descending order (desc c <-> asc n-1-c)
  if (tid == 0) {
    int r = n;
    if (a.mode == EIG_MODE_DECIDE) {
      const long long ncols = a.ncols_ptr ? (long long)a.ncols_mul * (*a.ncols_ptr) : a.ncols_const;
      int kmax = n < ncols ? n : (int)ncols;
      if (kmax < 1) kmax = 1;
      const double nrm2 = *a.norm2;
      const double tau2 = (a.dmodes > 1) ? a.eps * a.eps / (double)(a.dmodes - 1) * nrm2 : 0.0;
      double tail = 0.0;
      r = kmax;
      if (a.delta > 0.0) {
        // SV drop-off: the first lambda_{c+1} < delta^2 lambda_c
        const double d2 = a.delta * a.delta;
        for (int c = 1; c < kmax; ++c) {
          const double lp = (double)s_lam[n - c], lc = (double)s_lam[n - 1 - c];
          if (lp > 0.0 && (lc > 0.0 ? lc : 0.0) < d2 * lp) { r = c; break; }
        }
      }
      double margin = __longlong_as_double(0x7ff8000000000000LL);   // NaN: not an eps decision
      if (!(a.delta > 0.0) && a.eps > 0.0) {   // eps = 0: the cap alone (max rank TT-SVD)
        double kept = 0.0;
        bool stopped = false;
        for (int c = kmax - 1; c >= 1; --c) {
          const double l = (double)s_lam[n - 1 - c] * s_trace;
          tail += (l > 0.0 ? l : 0.0);
          if (tail <= tau2) { r = c; kept = tail; }
          else { stopped = true; break; }
        }
        if (tau2 > 0.0) margin = rank_margin(tau2, kept, tail, stopped);
      }
      if (a.rmax > 0 && r > a.rmax) { r = a.rmax; margin = __longlong_as_double(0x7ff8000000000000LL); }
      if (r < 1) r = 1;
      if (a.rank_out) *a.rank_out = r;
      if (a.margin_out) *a.margin_out = margin;
    }
    s_r = r;
    // clusters over the descending order: c joins c-1's cluster when close
    const float tn = fmaxf(fabsf(s_glo), fabsf(s_ghi));
    // clusters for Gram-Schmidt: gaps at which FP32 eigenvectors are not
    // resolved (eps ||T|| / gap of order one); wider gaps are handled by
    // the Newton-Schulz orthonormalisation below
    const float ortol = a.ortol_rel * tn;
    int cid = 0;
    for (int c = 0; c < n; ++c) {
      if (c > 0 && fabsf(s_lam[n - 1 - c] - s_lam[n - c]) > ortol) cid = c;
      s_clu[c] = cid;    // first member of c's cluster
    }
    const int nc = (a.mode == EIG_MODE_ALL) ? n : r;
    int cend = nc;
    for (int c = nc - 1; c >= 0; --c) {
      s_cend[c] = cend;  // one past the last member of c's cluster (among the copied)
      if (s_clu[c] == c) cend = c;
    }
  }
  __syncthreads();
  const int r = s_r;
  const int ncopy = (a.mode == EIG_MODE_ALL) ? n : r;
  if (a.sig_out)
    for (int c = tid; c < n; c += HT) a.sig_out[c] = (double)s_lam[n - 1 - c] * s_trace;

  HEEV_STAMP(3);
  // ---- 3. eigenvectors of T (descending order, one thread per vector)
  for (int c = tid; c < ncopy; c += HT)
    twisted_vector(s_d, s_e, n, s_lam[n - 1 - c], s_pivmin, Z + (size_t)ldz * c);
  __syncthreads();

  // ---- 4. orthogonalisation inside clusters, in descending order (the span
  // of the leading vectors of a cluster is kept).
  // 4a. modified Gram-Schmidt, right-looking, two sweeps: at step c every
  // warp loads z_c, forms q = z_c / |z_c| in registers (the same bits in
  // every warp: same data, same butterfly order) and removes q from its share
  // of the later members of c's cluster; one barrier per step, none for a
  // vector alone in its cluster.  A member whose residual norm in the first
  // sweep is below 1/4 is a degenerate copy (an exactly repeated eigenvalue,
  // e.g. the zero eigenvalues of a rank-deficient Gram, for which the twisted
  // factorisation returns the same vector): it projects nothing and is
  // replaced in 4b.
  HEEV_STAMP(4);
  int* bad = s_bad;
  for (int c = tid; c < ncopy; c += HT) bad[c] = 0;
  __syncthreads();
  for (int sweep = 0; sweep < 2; ++sweep) {
    for (int c = 0; c < ncopy; ++c) {
      const int cend = s_cend[c];
      if (cend - s_clu[c] <= 1) continue;                 // alone in its cluster (uniform)
      if (sweep == 1 && bad[c]) continue;                  // decided in sweep 0 (uniform)
      float q[4], nn = 0.f;
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const int i = lane + 32 * x;
        q[x] = (i < n) ? Z[i + (size_t)ldz * c] : 0.f;
        nn = fmaf(q[x], q[x], nn);
      }
      nn = warp_sum(nn);
      if (sweep == 0 && !(nn > 0.0625f)) {                 // uniform: every warp has nn
        if (tid == 0) bad[c] = 1;
        continue;
      }
      const float inv = rsqrtf(nn);
#pragma unroll
      for (int x = 0; x < 4; ++x) q[x] *= inv;
      if (tid == 0) s_inv[c] = inv;
      // four members per warp at a time: independent dot/butterfly chains
      for (int j0 = c + 1 + warp; j0 < cend; j0 += 4 * (HT / 32)) {
        float zr[4][4], h[4];
        bool act[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u * (HT / 32);
          act[u] = (j < cend) && !(sweep == 1 && bad[j]);
          h[u] = 0.f;
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            const int i = lane + 32 * x;
            zr[u][x] = (act[u] && i < n) ? Z[i + (size_t)ldz * j] : 0.f;
            h[u] = fmaf(q[x], zr[u][x], h[u]);
          }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
          for (int u = 0; u < 4; ++u) h[u] += __shfl_xor_sync(0xffffffffu, h[u], off);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (!act[u]) continue;
          float* zj = Z + (size_t)ldz * (j0 + u * (HT / 32));
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            const int i = lane + 32 * x;
            if (i < n) zj[i] = fmaf(-h[u], q[x], zr[u][x]);
          }
        }
      }
      __syncthreads();
    }
    // normalise what the sweep orthogonalised (z_c is not read again after
    // its own step, so the scaling waits until here)
    for (int c = warp; c < ncopy; c += HT / 32) {
      if (s_cend[c] - s_clu[c] <= 1 || bad[c]) continue;
      const float inv = s_inv[c];
      for (int i = lane; i < n; i += 32) Z[i + (size_t)ldz * c] *= inv;
    }
    __syncthreads();
  }

  if (a.phase_clk && tid == 0) {
    a.phase_clk[10] = clock64();
    int nb = 0, nm = 0;
    for (int c = 0; c < ncopy; ++c) {
      nb += bad[c];
      nm += (s_cend[c] - s_clu[c] > 1);
    }
    a.phase_clk[11] = nb;
    a.phase_clk[12] = nm;
  }
  // 4b. each degenerate copy becomes the unit vector e_i with the largest
  // component outside the span of the accepted vectors (residual
  // 1 - sum_j Z[i,j]^2; some e_i has at least (missing dimension)/n there),
  // orthogonalised twice against all accepted vectors (classical
  // Gram-Schmidt) and normalised; it is accepted from then on.
  float* coef = reinterpret_cast<float*>(s_p);   // s_p is free after step 1
  for (int c = 0; c < ncopy; ++c) {
    if (!bad[c]) continue;                               // uniform (smem flag)
    float best = -1.f;
    int bi = 0;
    for (int i = tid; i < n; i += HT) {
      float pr = 0.f;
      for (int j = 0; j < ncopy; ++j)
        if (j != c && !bad[j]) pr = fmaf(Z[i + (size_t)ldz * j], Z[i + (size_t)ldz * j], pr);
      const float res = 1.f - pr;
      if (res > best) { best = res; bi = i; }
    }
    // block argmax (ties: smallest index)
    for (int off = 16; off > 0; off >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { s_redf[warp] = best; s_pack[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      float bb = -1.f;
      int ii = 0;
      for (int w = 0; w < HT / 32; ++w)
        if (s_redf[w] > bb || (s_redf[w] == bb && s_pack[w] < ii)) { bb = s_redf[w]; ii = s_pack[w]; }
      s_pack[0] = ii;
    }
    __syncthreads();
    const int ui = s_pack[0];
    for (int i = tid; i < n; i += HT) Z[i + (size_t)ldz * c] = (i == ui) ? 1.f : 0.f;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = warp; j < ncopy; j += HT / 32) {
        float h = 0.f;
        const bool use = (j != c) && !bad[j];
        if (use)
          for (int i = lane; i < n; i += 32) h = fmaf(Z[i + (size_t)ldz * j], Z[i + (size_t)ldz * c], h);
        h = warp_sum(h);
        if (lane == 0) coef[j] = use ? h : 0.f;
      }
      __syncthreads();
      {
        // 4 partial sums per row (thread t: row t & 127, j = t >> 7 mod 4)
        const int i = tid & 127, ph = tid >> 7;
        float acc = 0.f;
        if (i < n)
          for (int j = ph; j < ncopy; j += 4) acc = fmaf(coef[j], Z[i + (size_t)ldz * j], acc);
        ((float*)s_part)[ph * HMAX + i] = acc;
      }
      __syncthreads();
      for (int i = tid; i < n; i += HT) {
        const float* pp = (const float*)s_part;
        Z[i + (size_t)ldz * c] -= pp[i] + pp[HMAX + i] + pp[2 * HMAX + i] + pp[3 * HMAX + i];
      }
      __syncthreads();
    }
    float part = 0.f;
    for (int i = tid; i < n; i += HT) {
      const float z = Z[i + (size_t)ldz * c];
      part = fmaf(z, z, part);
    }
    part = warp_sum(part);
    if (lane == 0) s_redf[warp] = part;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
      for (int w = 0; w < HT / 32; ++w) t += s_redf[w];
      bad[c] = 0;
      s_xn2 = (t > 0.f) ? rsqrtf(t) : 0.f;
    }
    __syncthreads();
    const float sc = s_xn2;
    if (sc > 0.f)
      for (int i = tid; i < n; i += HT) Z[i + (size_t)ldz * c] *= sc;
    __syncthreads();
  }

  HEEV_STAMP(5);
  if (hs.Z) {
    // split solve: the Newton-Schulz step and U = Q Z run in
    // heev_back_kernel over a cluster of CTAs
    for (int e = tid; e < n * ncopy; e += HT) hs.Z[e] = Z[(e % n) + (size_t)ldz * (e / n)];
    for (int k = warp; k < n - 2; k += HT / 32) {
      const int pk = k * (n - 2) - k * (k - 1) / 2;
      for (int i = k + 2 + lane; i < n; i += 32) hs.V[pk + (i - k - 2)] = A[i + (size_t)n * k];
    }
    for (int k = tid; k < n - 1; k += HT) hs.tau[k] = s_tau[k];
    if (tid == 0) hs.hdr[0] = ncopy;
    return;
  }
  // ---- 5. U = Q Z: compact the reflectors, then transform column chunks
  // packed reflector k (rows k+2..n-1) at offset P_k = sum_{k'<k} (n - k' - 2)
  const int npack = (n >= 2) ? (n - 2) * (n - 1) / 2 : 0;
  {
    float2 buf[16];
    int cnt = 0;
    for (int e = tid; e < npack && cnt < 16; e += HT, ++cnt) {
      // invert e -> (k, t): P_k <= e < P_{k+1}
      int k = 0, pk = 0;
      while (k < n - 2 && pk + (n - k - 2) <= e) { pk += n - k - 2; ++k; }
      const int i = k + 2 + (e - pk);
      buf[cnt] = A[i + (size_t)n * k];
    }
    __syncthreads();
    cnt = 0;
    for (int e = tid; e < npack && cnt < 16; e += HT, ++cnt) A[e] = buf[cnt];
    __syncthreads();
  }
  HEEV_STAMP(6);
  // ---- 4b. Newton-Schulz orthonormalisation Z <- Z (3 I - Z^T Z) / 2.
  // The vectors of distinct eigenvalues are orthogonal to O(eps ||T|| / gap)
  // (the accuracy order of any backward-stable solver); each step squares
  // the defect.  G = Z^T Z (dense) sits in the part of A freed by packing
  // the reflectors; the new Z passes through Uout (global, this kernel's own
  // output, overwritten by the back-transformation).  Both products use
  // 4 x 8 register tiles per thread.
  {
    float* Gd = reinterpret_cast<float*>(A + npack);             // ncopy x ncopy
    float* Zn = reinterpret_cast<float*>(a.Uout);                 // n x ncopy floats
    // tile: 4 rows spaced 32 apart (consecutive across the lanes of a warp)
    // x 8 columns (uniform across the warp: broadcast loads)
    const int nrb = (ncopy + 127) / 128, ncb = (ncopy + 7) / 8;
    for (int it = 0; it < a.ns_steps; ++it) {
      // G = Z^T Z
      for (int t = warp; t < nrb * ncb; t += HT / 32) {
        const int i0 = (t % nrb) * 128 + lane, j0 = (t / nrb) * 8;
        float acc[4][8];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 8; ++y) acc[x][y] = 0.f;
        for (int l = 0; l < n; ++l) {
          float zi[4], zj[8];
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            const int i = i0 + 32 * x;
            zi[x] = (i < ncopy) ? Z[l + (size_t)ldz * i] : 0.f;
          }
#pragma unroll
          for (int y = 0; y < 8; ++y) zj[y] = (j0 + y < ncopy) ? Z[l + (size_t)ldz * (j0 + y)] : 0.f;
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(zi[x], zj[y], acc[x][y]);
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 8; ++y) {
            const int i = i0 + 32 * x;
            if (i < ncopy && j0 + y < ncopy) Gd[i + (size_t)ncopy * (j0 + y)] = acc[x][y];
          }
      }
      __syncthreads();

      // Zn = 1.5 Z - 0.5 Z G
      const int nrz = (n + 127) / 128;
      for (int t = warp; t < nrz * ncb; t += HT / 32) {
        const int i0 = (t % nrz) * 128 + lane, c0 = (t / nrz) * 8;
        float acc[4][8];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 8; ++y) acc[x][y] = 0.f;
        for (int l = 0; l < ncopy; ++l) {
          float zl[4], gl[8];
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            const int i = i0 + 32 * x;
            zl[x] = (i < n) ? Z[i + (size_t)ldz * l] : 0.f;
          }
#pragma unroll
          for (int y = 0; y < 8; ++y) gl[y] = (c0 + y < ncopy) ? Gd[l + (size_t)ncopy * (c0 + y)] : 0.f;
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(zl[x], gl[y], acc[x][y]);
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 8; ++y) {
            const int i = i0 + 32 * x, c = c0 + y;
            if (i < n && c < ncopy) Zn[i + (size_t)n * c] = 1.5f * Z[i + (size_t)ldz * c] - 0.5f * acc[x][y];
          }
      }
      __syncthreads();
      for (int e = tid; e < n * ncopy; e += HT) Z[(e % n) + (size_t)ldz * (e / n)] = Zn[e];
      __syncthreads();
    }
  }
  HEEV_STAMP(7);
  if (a.orth_flag) {
    // orthonormality after Newton-Schulz: a spectrum degenerate at FP32
    // resolution can leave a cluster that neither the Gram-Schmidt nor the
    // Newton-Schulz steps repair; such a solve is redone by the Jacobi
    // solver that the host queues behind this kernel, gated by the flag
    for (int e = tid; e < ncopy * ncopy; e += HT) {
      const int i = e % ncopy, j = e / ncopy;
      if (j < i) continue;
      float g = 0.f;
      for (int l = 0; l < n; ++l) g = fmaf(Z[l + (size_t)ldz * i], Z[l + (size_t)ldz * j], g);
      if (i == j) g -= 1.f;
      if (!(fabsf(g) <= 1e-4f)) atomicExch(a.orth_flag, 1);   // NaN included
    }
  }
  float2* Vp = A;                                  // packed reflectors
  float2* Uc = A + npack;                          // column chunk after them
  // columns per chunk: what fits in the rest of the n x n region, at most 64
  // (the back-transformation maps 8 threads to a column); leading dimension
  // n + 1 keeps the 4 column groups of a warp on different banks
  const int ldu = n + 1;
  const int cw = max(1, min(64, (n * n - npack) / ldu));
  for (int cb = 0; cb < ncopy; cb += cw) {
    const int nc = min(cw, ncopy - cb);
    for (int c = tid >> 7; c < nc; c += HT / 128)
      for (int i = tid & 127; i < n; i += 128) Uc[i + (size_t)ldu * c] = make_float2(Z[i + (size_t)ldz * (cb + c)], 0.f);
    __syncthreads();
    // 8 threads per column; the group owns the column for all reflectors.
    // The 4 groups of a warp take columns 8 apart: with ldu = n + 1 (n even)
    // their 16-word windows then start 16 banks apart (2 wavefronts per warp
    // access, the minimum for 32 float2)
    const int grp = tid >> 3, sub = tid & 7, gw = grp >> 2;
    const int c = (gw & 7) + 8 * (grp & 3) + 32 * (gw >> 3);
    if (c < nc) {
      float2* u = Uc + (size_t)ldu * c;
      for (int k = n - 2; k >= 0; --k) {
        const float2 tau = s_tau[k];
        if (tau.x == 0.f && tau.y == 0.f) continue;
        const int pk = k * (n - 2) - k * (k - 1) / 2;   // sum_{k'<k} (n - k' - 2)
        float2 w = make_float2(0.f, 0.f);
        for (int i = k + 1 + sub; i < n; i += 8) {
          const float2 v = (i == k + 1) ? make_float2(1.f, 0.f) : Vp[pk + (i - k - 2)];
          const float2 ui = u[i];
          w.x = fmaf(v.x, ui.x, fmaf(v.y, ui.y, w.x));   // conj(v) u
          w.y = fmaf(v.x, ui.y, fmaf(-v.y, ui.x, w.y));
        }
        const unsigned gm = 0xffu << (lane & ~7);
        w.x += __shfl_xor_sync(gm, w.x, 1);
        w.y += __shfl_xor_sync(gm, w.y, 1);
        w.x += __shfl_xor_sync(gm, w.x, 2);
        w.y += __shfl_xor_sync(gm, w.y, 2);
        w.x += __shfl_xor_sync(gm, w.x, 4);
        w.y += __shfl_xor_sync(gm, w.y, 4);
        const float2 f = cmulf(tau, w);
        for (int i = k + 1 + sub; i < n; i += 8) {
          const float2 v = (i == k + 1) ? make_float2(1.f, 0.f) : Vp[pk + (i - k - 2)];
          float2 ui = u[i];
          ui.x -= v.x * f.x - v.y * f.y;
          ui.y -= v.x * f.y + v.y * f.x;
          u[i] = ui;
        }
        __syncwarp(gm);
      }
    }
    __syncthreads();
    for (int c = tid >> 7; c < nc; c += HT / 128)
      for (int i = tid & 127; i < n; i += 128) a.Uout[(size_t)n * (cb + c) + i] = Uc[i + (size_t)ldu * c];
    __syncthreads();
  }
  __syncthreads();
  HEEV_STAMP(8);
  if (a.core_out) {
    if (a.U1) {
      for (int e = tid; e < n * r; e += HT) {
        const int i = e % n, c = e / n;
        KAcc32 acc;
        for (int l = 0; l < n; ++l) acc.add_mul(a.U1[i + (size_t)n * l], a.Uout[l + (size_t)n * c]);
        a.core_out[e] = acc.get();
      }
    } else if (a.core_out != a.Uout) {
      for (int e = tid; e < n * r; e += HT) a.core_out[e] = a.Uout[e];
    }
  }
  HEEV_STAMP(9);
}

// ---------------------------------------------------------------------------
// Second half of a split solve, over a cluster of HB_CTAS CTAs (one SM each):
// every CTA holds all of Z and owns a slice of at most 16 columns.
//   Newton-Schulz, 3 steps: G_s = Z^T Z_s, Z'_s = 1.5 Z_s - 0.5 Z G_s for the
//     own slice s, then Z'_s is stored into every CTA's second Z buffer
//     (distributed shared memory) and the cluster synchronises;
//   U_s = Q Z_s: the reflectors, newest first, on the own columns, the
//     column held in registers by 16 threads (8 rows each, fixed ownership:
//     no barrier between reflectors);
//   optionally core_s = U1 U_s for the kept columns.
// The column products reduce in the same order as the one-CTA kernel's tiles.
constexpr int HB_CTAS = 8;
constexpr int HB_THREADS = 256;

__global__ void __cluster_dims__(HB_CTAS, 1, 1) __launch_bounds__(HB_THREADS)
    heev_back_kernel(EigArgs<float2> a, HeevSplit hs, int mg_cap) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float2 s_tau[HMAX];
  const int tid = threadIdx.x, lane = tid & 31;
  const int rank = (int)cluster.block_rank();
  const long long t0 = clock64();
  const int n = a.mg_ptr ? a.mg_mul * (*a.mg_ptr) : a.mg_const;
  const int ncopy = hs.hdr[0];
  const int ldz = n + 1;
  const size_t zcap = (size_t)mg_cap * (mg_cap + 1);
  float* Zb0 = reinterpret_cast<float*>(smem_raw);
  float* Zb1 = Zb0 + zcap;
  float2* Vp = reinterpret_cast<float2*>(Zb1 + zcap);
  const int npack = (n >= 2) ? (n - 2) * (n - 1) / 2 : 0;
  const int nvcap = (mg_cap >= 2) ? (mg_cap - 2) * (mg_cap - 1) / 2 : 0;
  float2* Uc = Vp + nvcap;                       // 16 x (n + 1) float2 (also G_s)
  float* Gs = reinterpret_cast<float*>(Uc);      // ncopy x 16 floats, ld ncopy

  const int cw = (ncopy + HB_CTAS - 1) / HB_CTAS;  // <= 16
  const int c0 = rank * cw;
  const int nc = max(0, min(cw, ncopy - c0));

  for (int e = tid; e < n * ncopy; e += HB_THREADS) Zb0[(e % n) + (size_t)ldz * (e / n)] = hs.Z[e];
  for (int e = tid; e < npack; e += HB_THREADS) Vp[e] = hs.V[e];
  for (int k = tid; k < n - 1; k += HB_THREADS) s_tau[k] = hs.tau[k];
  cluster.sync();   // every CTA has started and loaded (remote stores follow)
  const long long t1 = clock64();

  float* Z = Zb0;
  float* Zn = Zb1;
  // thread -> (row i = tid & 127, columns jg, jg + 2, ..., jg + 14)
  const int ti = tid & 127, jg = tid >> 7;
  for (int it = 0; it < a.ns_steps; ++it) {
    for (int i = ti; i < ncopy; i += 128) {
      float acc[8];
#pragma unroll
      for (int y = 0; y < 8; ++y) acc[y] = 0.f;
      for (int l = 0; l < n; ++l) {
        const float zi = Z[l + (size_t)ldz * i];
#pragma unroll
        for (int y = 0; y < 8; ++y) {
          const int j = jg + 2 * y;
          const float zj = (j < nc) ? Z[l + (size_t)ldz * (c0 + j)] : 0.f;
          acc[y] = fmaf(zi, zj, acc[y]);
        }
      }
#pragma unroll
      for (int y = 0; y < 8; ++y) {
        const int j = jg + 2 * y;
        if (j < nc) Gs[i + (size_t)ncopy * j] = acc[y];
      }
    }
    __syncthreads();
    for (int i = ti; i < n; i += 128) {
      float acc[8];
#pragma unroll
      for (int y = 0; y < 8; ++y) acc[y] = 0.f;
      for (int l = 0; l < ncopy; ++l) {
        const float zl = Z[i + (size_t)ldz * l];
#pragma unroll
        for (int y = 0; y < 8; ++y) {
          const int j = jg + 2 * y;
          const float g = (j < nc) ? Gs[l + (size_t)ncopy * j] : 0.f;
          acc[y] = fmaf(zl, g, acc[y]);
        }
      }
#pragma unroll
      for (int y = 0; y < 8; ++y) {
        const int j = jg + 2 * y;
        if (j < nc) acc[y] = 1.5f * Z[i + (size_t)ldz * (c0 + j)] - 0.5f * acc[y];
      }
      for (int dst = 0; dst < HB_CTAS; ++dst) {
        float* Zr = cluster.map_shared_rank(Zn, dst);
#pragma unroll
        for (int y = 0; y < 8; ++y) {
          const int j = jg + 2 * y;
          if (j < nc) Zr[i + (size_t)ldz * (c0 + j)] = acc[y];
        }
      }
    }
    cluster.sync();   // all slices stored everywhere; the old buffer is free
    float* t = Z;
    Z = Zn;
    Zn = t;
  }
  const long long t2 = clock64();

  // U_s = Q Z_s; thread (column cc = tid >> 4, sub = tid & 15) owns rows
  // sub + 16 m
  const int cc = tid >> 4, sub = tid & 15;
  float2 u[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int i = sub + 16 * m;
    u[m] = make_float2((cc < nc && i < n) ? Z[i + (size_t)ldz * (c0 + cc)] : 0.f, 0.f);
  }
  const unsigned gm = 0xffffu << (lane & 16);
  for (int k = n - 2; k >= 0; --k) {
    const float2 tau = s_tau[k];
    if (tau.x == 0.f && tau.y == 0.f) continue;
    const int pk = k * (n - 2) - k * (k - 1) / 2;
    float2 v[8];
    float2 w = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int i = sub + 16 * m;
      v[m] = (i == k + 1) ? make_float2(1.f, 0.f)
             : (i > k + 1 && i < n) ? Vp[pk + (i - k - 2)] : make_float2(0.f, 0.f);
      w.x = fmaf(v[m].x, u[m].x, fmaf(v[m].y, u[m].y, w.x));   // conj(v) u
      w.y = fmaf(v[m].x, u[m].y, fmaf(-v[m].y, u[m].x, w.y));
    }
#pragma unroll
    for (int off = 1; off < 16; off <<= 1) {
      w.x += __shfl_xor_sync(gm, w.x, off);
      w.y += __shfl_xor_sync(gm, w.y, off);
    }
    const float2 f = cmulf(tau, w);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      u[m].x -= v[m].x * f.x - v[m].y * f.y;
      u[m].y -= v[m].x * f.y + v[m].y * f.x;
    }
  }
  const long long t3 = clock64();
  if (cc < nc) {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int i = sub + 16 * m;
      if (i < n) a.Uout[(size_t)n * (c0 + cc) + i] = u[m];
    }
  }
  if (a.core_out) {
    const int r = ncopy;   // all columns (MODE_ALL) or the decided rank
    if (a.U1) {
      // Gs is free: stage the own columns, ld n + 1
      if (cc < nc) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int i = sub + 16 * m;
          if (i < n) Uc[i + (size_t)ldz * cc] = u[m];
        }
      }
      __syncthreads();
      for (int e = tid; e < n * nc; e += HB_THREADS) {
        const int i = e % n, c = e / n;
        if (c0 + c >= r) continue;
        KAcc32 acc;
        for (int l = 0; l < n; ++l) acc.add_mul(a.U1[i + (size_t)n * l], Uc[l + (size_t)ldz * c]);
        a.core_out[i + (size_t)n * (c0 + c)] = acc.get();
      }
    } else if (a.core_out != a.Uout && cc < nc && c0 + cc < r) {
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int i = sub + 16 * m;
        if (i < n) a.core_out[(size_t)n * (c0 + cc) + i] = u[m];
      }
    }
  }
  if (a.phase_clk && rank == 0 && tid == 0) {
    // this SM's clock differs from the first kernel's: durations are added
    // to the first kernel's last stamp
    const long long p5 = a.phase_clk[5];
    a.phase_clk[6] = p5 + (t1 - t0);
    a.phase_clk[7] = p5 + (t2 - t0);
    a.phase_clk[8] = p5 + (t3 - t0);
    a.phase_clk[9] = p5 + (clock64() - t0);
  }
}

size_t heev_tri_smem_bytes(int mg_cap) {
  return (size_t)mg_cap * mg_cap * sizeof(float2) + (size_t)mg_cap * (mg_cap + 1) * sizeof(float);
}

static size_t heev_back_smem_bytes(int mg_cap) {
  const size_t nv = (mg_cap >= 2) ? (size_t)(mg_cap - 2) * (mg_cap - 1) / 2 : 0;
  const size_t gs = std::max((size_t)16 * (mg_cap + 1) * sizeof(float2), (size_t)16 * mg_cap * sizeof(float));
  return 2 * (size_t)mg_cap * (mg_cap + 1) * sizeof(float) + nv * sizeof(float2) + gs;
}

static float g_heev_ortol = 1e-6f;
static int g_heev_ns = 3;

void heev_set_cluster_params(double ortol_rel, int ns_steps) {
  g_heev_ortol = ortol_rel > 0.0 ? (float)ortol_rel : 1e-6f;
  g_heev_ns = ns_steps > 0 ? ns_steps : 3;
}

void launch_heev_tri(const EigArgs<float2>& a_in, int mg_cap, cudaStream_t s) {
  EigArgs<float2> a = a_in;
  a.ortol_rel = g_heev_ortol;
  a.ns_steps = g_heev_ns;
  static std::atomic<unsigned long long> configured{0};
  if (first_on_device(&configured)) {
    cudaFuncSetAttribute(heev_tri_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)heev_tri_smem_bytes(HMAX));
    cudaFuncSetAttribute(heev_back_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)heev_back_smem_bytes(HMAX));
  }
  HeevSplit hs{nullptr, nullptr, nullptr, nullptr};
  void* buf = nullptr;
  if (mg_cap > 32) {
    // Z (floats) | reflectors | tau | header
    auto al16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    const size_t zb = al16((size_t)mg_cap * mg_cap * sizeof(float));
    const size_t vb = al16((size_t)mg_cap * mg_cap / 2 * sizeof(float2));
    const size_t tb = al16((size_t)mg_cap * sizeof(float2));
    buf = scratch_alloc(zb + vb + tb + 16, s);
    if (buf) {
      char* p = (char*)buf;
      hs.Z = (float*)p;
      hs.V = (float2*)(p + zb);
      hs.tau = (float2*)(p + zb + vb);
      hs.hdr = (int*)(p + zb + vb + tb);
    }
  }
  heev_tri_kernel<<<1, HT, heev_tri_smem_bytes(mg_cap), s>>>(a, hs);
  if (buf) {
    heev_back_kernel<<<HB_CTAS, HB_THREADS, heev_back_smem_bytes(mg_cap), s>>>(a, hs, mg_cap);
    scratch_free(buf, s);
  }
}

}  // namespace qtt
