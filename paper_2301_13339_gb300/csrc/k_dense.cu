// Dense building blocks of the large-rank rounding (ranks above 64):
//
//  * big_qr_q  -- blocked Householder QR of an m x n matrix held in global
//    memory (m <= BQ_MAXM) and the formation of the first nq columns of Q.
//    Panels of BQ_NB columns are factored by one CTA in shared memory
//    (LAPACK's H_k = I - tau_k v_k v_k^H, v_k = [1; A[k+1:, k]]), their
//    compact-WY factor T (H_1 ... H_nb = I - V T V^H, upper triangular) is
//    formed in the same CTA; the next panel's columns receive it inside the
//    next panel's kernel and the other trailing columns from many CTAs on a
//    side stream (Q^H = I - V T^H V^H, 8 columns per CTA, V staged in shared
//    memory).  Q = H_1 ... H_k [I; 0] is then accumulated in one launch,
//    each CTA carrying two columns through every panel from the last one.
//    Householder QR keeps Q orthonormal to working precision also when A is
//    rank deficient, which the randomised range finder of the rounding needs.
//
//  * cgemm      -- C = op(A) B for complex64 B and C and a complex64 or real
//    A, any strides (unit stride along the rows of A or along k; along k for
//    B; along the rows of C), batched over a two-level batch index.  64 x 64
//    output tiles, 16-deep k chunks staged in shared memory, 4 x 4 outputs
//    per thread, one CTA per SM; each chunk is summed with plain FMAs and
//    added to the running sum with compensation (Kahan), so long
//    contractions keep about one rounding error per chunk instead of one
//    per term.
#include "qtt_internal.cuh"
#include "house_qr.cuh"
#include <algorithm>
#include <atomic>

namespace qtt {

// ---------------------------------------------------------------- QR
// panel width: the one-CTA panel factorisation issues ~kb^2 M instructions
// per panel, so the panel chain of a QR costs ~kb n M and a narrower panel
// moves work to the many-CTA block-reflector updates
constexpr int BQ_NB = 16;
constexpr int BQ_CB = 8;         // columns per CTA in the block-reflector application
constexpr int BQ_MAXM = 1024;    // rows (panel in shared memory: 1024 x 16 x 8 B)

// Factor the panel A[p:m, p:p+kb] (kb <= BQ_NB) in shared memory (ld odd,
// so consecutive columns fall on different banks), write it back (R on and
// above the diagonal, the v_k below), V^T (kb x mp, row a = v_a, unit
// diagonal and zeros above it written out) to Vt, and T (BQ_NB x BQ_NB,
// column-major) to Tm.
//
// WPC (1 or 2) warps per trailing column, each over every WPC-th 32-row
// stripe, and one barrier per reflector: the warps that update column k + 1
// in step k also measure its largest entry and scaled sum of squares and,
// before the step's barrier, derive reflector k + 1 from them (tau, the
// scale 1/(alpha - beta) of v, beta), which every warp reads in step k + 1
// (look-ahead); the trailing update takes v_i = col_i * scal on the fly
// (v^H x = x_k + conj(scal) sum_{i>k} conj(col_i) x_i; with WPC = 2 the two
// warps' partial sums are added in a fixed order after a 64-thread barrier
// of the pair), so column k is scaled into v only in the next step, by the
// last warp, which no trailing column needs.  The library launches
// WPC = 1: two warps per column halve each warp's chain but duplicate its
// fixed work, and measured slower on every panel height of the rounding
// (up to 1024 rows).
constexpr int BQP_THREADS = 1024;
// the pairs of the trailing columns use warps 0 .. 2 (BQ_NB - 1) - 1 and
// named barriers 1 .. BQ_NB - 1; the last warp scales the finished column
static_assert(2 * (BQ_NB - 1) < BQP_THREADS / 32 - 1 && BQ_NB - 1 <= 15, "panel warp layout");

// largest |re|, |im| of x over rows i >= i0, and sum over i > i0 of
// |x_i / amax|^2 (all lanes of the warp get both)
template <typename T>
__device__ __forceinline__ void bq_col_norm(const T* x, int i0, int mp, int lane,
                                            typename Sc<T>::R& amax, typename Sc<T>::R& ssq) {
  using R = typename Sc<T>::R;
  R a = (R)0;
  for (int i = i0 + lane; i < mp; i += 32) a = rmax(a, rmax(rabs(sreal(x[i])), rabs(simag(x[i]))));
  for (int off = 16; off > 0; off >>= 1) a = rmax(a, __shfl_xor_sync(0xffffffffu, a, off));
  R q = (R)0;
  if (a > (R)0) {
    const R inv = (R)1 / a;
    for (int i = i0 + 1 + lane; i < mp; i += 32) q += sabs2(rscale(x[i], inv));
  }
  for (int off = 16; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
  amax = a;
  ssq = q;
}

// Householder reflector of a column from its largest entry amax (of |re|,
// |im| over the rows from the diagonal on), the scaled sum of squares part
// below the diagonal and the diagonal entry alpha: tau, the scale
// 1 / (alpha - beta) of v and beta, computed at the column's scale (no
// overflow or underflow of |alpha - beta|^2 at any data scale)
template <typename T>
__device__ __forceinline__ void bq_reflector(typename Sc<T>::R amax, typename Sc<T>::R part, T alpha,
                                             T& tau_o, T& scal_o, T& beta_o) {
  using R = typename Sc<T>::R;
  T tau = szero<T>(), scal = szero<T>(), beta_s = alpha;
  if (amax > (R)0) {
    const R inv = (R)1 / amax;
    const T al = rscale(alpha, inv);
    const R ax = sreal(al), ay = simag(al);
    if (part > (R)0 || ay != (R)0) {
      const R nrm = sqrt(ax * ax + ay * ay + part);
      const R beta = (ax >= (R)0) ? -nrm : nrm;
      const R rb = (R)1 / beta;
      tau = make_scalar<T>((beta - ax) * rb, -ay * rb);
      const R dr = ax - beta, di = ay, rden = (R)1 / (dr * dr + di * di);
      scal = rscale(make_scalar<T>(dr * rden, -di * rden), inv);   // 1 / (alpha - beta)
      beta_s = make_scalar<T>(beta * amax, (R)0);
    }
  }
  tau_o = tau;
  scal_o = scal;
  beta_o = beta_s;
}

__device__ __forceinline__ void bq_pair_sync(int pair) {
  asm volatile("bar.sync %0, 64;" ::"r"(pair + 1) : "memory");
}

template <typename T, int WPC>
__global__ void __launch_bounds__(BQP_THREADS)
k_bq_panel(T* __restrict__ A, int m, int p, int kb, T* __restrict__ Tm, T* __restrict__ Vt,
           const T* __restrict__ Vprev, const T* __restrict__ Tprev, int kbp) {
  static_assert(WPC == 1 || WPC == 2, "warps per column");
  using R = typename Sc<T>::R;
  extern __shared__ __align__(16) unsigned char bq_smem[];
  // with Vprev the panel's columns first receive the block reflector of the
  // previous panel (rows p - kbp .. m - 1, V^T = Vprev, T = Tprev): the
  // buffer holds those rows, P is its part from row p on
  const int off = Vprev ? kbp : 0;
  T* Xb = reinterpret_cast<T*>(bq_smem);
  T* P = Xb + off;
  __shared__ T s_tau[BQ_NB], s_scal[BQ_NB], s_beta[BQ_NB];
  __shared__ R s_lam[BQ_NB][2], s_lsq[BQ_NB][2];   // look-ahead partials of each half
  __shared__ T s_pd[BQ_NB][2];                      // partial dots of each pair
  __shared__ T s_Y[BQ_NB * BQ_NB];
  __shared__ T s_T[BQ_NB * BQ_NB];
  __shared__ R s_wmax[BQP_THREADS / 32];
  const int mp = m - p;
  const int mpp = mp + off;
  const int ld = mpp | 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = warp / WPC, half = warp % WPC;
  // element loops: warp w takes column w / 2 (and + 16) and every other
  // 32-row stripe
  const int ec = warp >> 1, er = lane + 32 * (warp & 1);
  for (int j = ec; j < kb; j += 16)
    for (int i = er; i < mpp; i += 64) Xb[i + (size_t)ld * j] = A[(size_t)(p - off + i) + (size_t)m * (p + j)];
  for (int e = tid; e < BQ_NB * BQ_NB; e += BQP_THREADS) {
    s_T[e] = szero<T>();
    s_Y[e] = szero<T>();
  }
  if (tid < 2 * BQ_NB) {
    (&s_lam[0][0])[tid] = (R)0;
    (&s_lsq[0][0])[tid] = (R)0;
  }
  __syncthreads();
  if (off > 0) {
    // X <- (I - V T^H V^H) X with the arithmetic of bq_apply_staged (per
    // column the same sums in the same order): W = V^H X, one warp per
    // (reflector, 8 columns), lanes over the rows; W2 = T^H W; then each
    // thread updates its rows of all columns.  s_Y and s_T serve as W and
    // W2 (they are zeroed again before the factorisation uses them).
    T* sW = s_Y;    // W[a][j] at a + BQ_NB j
    T* sW2 = s_T;
    {
      const int a = warp % BQ_NB, cb = (warp / BQ_NB) * 8;
      if (a < kbp && cb < kb) {
        T acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = szero<T>();
        // four rows' V entries in flight per lane (the loads come from L2),
        // each row then added in row order
        int i = lane;
        for (; i + 96 < mpp; i += 128) {
          T v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = Vprev[i + 32 * u + (size_t)mpp * a];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c)
              if (cb + c < kb) macc(acc[c], v[u], Xb[i + 32 * u + (size_t)ld * (cb + c)]);
        }
        for (; i < mpp; i += 32) {
          const T v = Vprev[i + (size_t)mpp * a];
#pragma unroll
          for (int c = 0; c < 8; ++c)
            if (cb + c < kb) macc(acc[c], v, Xb[i + (size_t)ld * (cb + c)]);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const T w = warp_sum(acc[c]);
          if (lane == 0 && cb + c < kb) sW[a + BQ_NB * (cb + c)] = w;
        }
      }
    }
    __syncthreads();
    if (tid < BQ_NB * BQ_NB) {
      const int a = tid % BQ_NB, c = tid / BQ_NB;
      T w2 = szero<T>();
      if (a < kbp && c < kb)
        for (int b = 0; b <= a; ++b) macc(w2, Tprev[b + BQ_NB * a], sW[b + BQ_NB * c]);
      sW2[a + BQ_NB * c] = w2;
    }
    __syncthreads();
    for (int i = tid; i < mpp; i += BQP_THREADS) {
      T v[BQ_NB];
#pragma unroll
      for (int a = 0; a < BQ_NB; ++a) v[a] = (a < kbp) ? Vprev[i + (size_t)mpp * a] : szero<T>();
      for (int j = 0; j < kb; ++j) {
        T sacc = szero<T>();
#pragma unroll
        for (int a = 0; a < BQ_NB; ++a)
          if (a < kbp) mac(sacc, v[a], sW2[a + BQ_NB * j]);
        Xb[i + (size_t)ld * j] = ssub(Xb[i + (size_t)ld * j], sacc);
      }
    }
    __syncthreads();
    for (int e = tid; e < BQ_NB * BQ_NB; e += BQP_THREADS) {
      s_T[e] = szero<T>();
      s_Y[e] = szero<T>();
    }
  }
  {
    R lmax = (R)0;
    for (int j = ec; j < kb; j += 16)
      for (int i = er; i < mp; i += 64) {
        const T v = P[i + (size_t)ld * j];
        lmax = rmax(lmax, rmax(rabs(sreal(v)), rabs(simag(v))));
      }
    for (int o = 16; o > 0; o >>= 1) lmax = rmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if (lane == 0) s_wmax[warp] = lmax;
  }
  __syncthreads();
  // A panel whose largest entry lies outside [2^-E, 2^E] (E = 30 in FP32,
  // 200 in FP64) is factored scaled by a power of two near its inverse:
  // the dot products of the trailing updates multiply two entries and would
  // under- or overflow.  Householder QR is homogeneous (v, tau and T do
  // not depend on the scale, R scales with it), so only R is scaled back
  // when the panel is written out; panels inside the range are untouched.
  int pexp = 0;
  {
    R pm = (R)0;
    for (int w = 0; w < BQP_THREADS / 32; ++w) pm = rmax(pm, s_wmax[w]);
    const int E = sizeof(R) == 4 ? 30 : 200;
    if (pm > (R)0 && pm < (R)INFINITY) {
      const int e = ilogb(pm);
      if (e < -E || e > E) pexp = e;
    }
  }
  if (pexp != 0) {   // block-uniform
    for (int j = ec; j < kb; j += 16)
      for (int i = er; i < mp; i += 64) {
        T& v = P[i + (size_t)ld * j];
        v = make_scalar<T>(scalbn(sreal(v), -pexp), scalbn(simag(v), -pexp));
      }
    __syncthreads();
  }
  const int kmax = min(mp, kb);
  // the unscaled look-ahead sum is exact enough wherever amax^2 neither
  // overflows nor underflows; outside that range the column is measured
  // again with the scaled two-pass sum
  const R lo = sizeof(R) == 4 ? (R)1e-15 : (R)1e-140, hi = sizeof(R) == 4 ? (R)1e15 : (R)1e140;
  if (warp == 0 && kmax > 0) {
    R a, q;
    bq_col_norm(P, 0, mp, lane, a, q);
    if (lane == 0) bq_reflector(a, q, P[0], s_tau[0], s_scal[0], s_beta[0]);
  }
  __syncthreads();
  constexpr int RS = 32 * WPC;   // row stride of a warp
  for (int k = 0; k < kmax; ++k) {
    const T* col = P + (size_t)ld * k;
    const int nt = kb - 1 - k;   // trailing columns of the panel (<= 15)
    if (grp < nt) {
      const T tau = s_tau[k], scal = s_scal[k];
      {
        // x <- (I - conj(tau) v v^H) x for trailing column j over the rows
        // k + 1 + 32 half + RS t + lane; four stripes per lane in flight
        const int j = k + 1 + grp;
        T* x = P + (size_t)ld * j;
        T a0 = szero<T>(), a1 = szero<T>(), a2 = szero<T>(), a3 = szero<T>();
        const int r0 = k + 1 + 32 * half + lane;
        int i = r0;
        for (; i + 3 * RS < mp; i += 4 * RS) {
          const T c0 = col[i], c1 = col[i + RS], c2 = col[i + 2 * RS], c3 = col[i + 3 * RS];
          const T x0 = x[i], x1 = x[i + RS], x2 = x[i + 2 * RS], x3 = x[i + 3 * RS];
          macc(a0, c0, x0);
          macc(a1, c1, x1);
          macc(a2, c2, x2);
          macc(a3, c3, x3);
        }
        for (; i < mp; i += RS) macc(a0, col[i], x[i]);
        const T pdot = warp_sum(sadd(sadd(a0, a1), sadd(a2, a3)));
        const T xk = x[k];
        T sdot = pdot;
        if (WPC == 2) {
          if (lane == 0) s_pd[grp][half] = pdot;
          bq_pair_sync(grp);            // both partials written, both halves have read x[k]
          sdot = sadd(s_pd[grp][0], s_pd[grp][1]);
        } else {
          __syncwarp();                 // every lane has read x[k]
        }
        const T wdot = sadd(xk, smul(conjg(scal), sdot));
        const T f = smul(conjg(tau), wdot);
        const T fs = smul(scal, f);
        if (half == 0 && lane == 0) x[k] = ssub(xk, f);
        // column k + 1 (the next reflector's) also measures itself while it
        // is updated: largest |re|, |im| over rows >= k + 1 and the plain
        // sum of squares below row k + 1, per warp; then its warps derive
        // reflector k + 1 for the next step
        const bool look = (j == k + 1 && j < kmax);
        R am = (R)0, sq = (R)0;
        int r = r0;
        for (; r + 3 * RS < mp; r += 4 * RS) {
          T y[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) y[u] = ssub(x[r + RS * u], smul(col[r + RS * u], fs));
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            x[r + RS * u] = y[u];
            if (look) {
              am = rmax(am, rmax(rabs(sreal(y[u])), rabs(simag(y[u]))));
              if (r + RS * u > j) sq += sabs2(y[u]);
            }
          }
        }
        for (; r < mp; r += RS) {
          const T y = ssub(x[r], smul(col[r], fs));
          x[r] = y;
          if (look) {
            am = rmax(am, rmax(rabs(sreal(y)), rabs(simag(y))));
            if (r > j) sq += sabs2(y);
          }
        }
        if (look) {
          for (int o = 16; o > 0; o >>= 1) {
            am = rmax(am, __shfl_xor_sync(0xffffffffu, am, o));
            sq += __shfl_xor_sync(0xffffffffu, sq, o);
          }
          if (lane == 0) { s_lam[j][half] = am; s_lsq[j][half] = sq; }
          if (WPC == 2) bq_pair_sync(grp);   // both halves measured and updated
          else __syncwarp();
          if (half == 0) {
            // the halves combined in a fixed order
            R amax = rmax(s_lam[j][0], s_lam[j][1]), part;
            if (amax == (R)0 || (amax > lo && amax < hi)) {
              part = (amax > (R)0) ? (s_lsq[j][0] + s_lsq[j][1]) / (amax * amax) : (R)0;
            } else {
              bq_col_norm(x, j, mp, lane, amax, part);
            }
            if (lane == 0) bq_reflector(amax, part, x[j], s_tau[j], s_scal[j], s_beta[j]);
          }
        }
      }
    } else if (warp == BQP_THREADS / 32 - 1 && k > 0) {
      // column k - 1 is final: v_{k-1} = col * scal below the diagonal, beta on it
      T* c1 = P + (size_t)ld * (k - 1);
      const T sc = s_scal[k - 1];
      for (int r = k + lane; r < mp; r += 32) c1[r] = smul(c1[r], sc);
      if (lane == 0) c1[k - 1] = s_beta[k - 1];
    }
    __syncthreads();
  }
  if (warp == 0 && kmax > 0) {
    T* c1 = P + (size_t)ld * (kmax - 1);
    const T sc = s_scal[kmax - 1];
    for (int r = kmax + lane; r < mp; r += 32) c1[r] = smul(c1[r], sc);
    if (lane == 0) c1[kmax - 1] = s_beta[kmax - 1];
  }
  __syncthreads();
  // Y[a + NB b] = v_a^H v_b (a < b), one warp per pair, lanes over the rows
  // i > b (row b: v_b = 1)
  for (int pr = warp; pr < kmax * kmax; pr += BQP_THREADS / 32) {
    const int a = pr % kmax, b = pr / kmax;
    if (a >= b) continue;   // warp-uniform
    const T* va = P + (size_t)ld * a;
    const T* vb = P + (size_t)ld * b;
    T acc = szero<T>();
    for (int i = b + 1 + lane; i < mp; i += 32) macc(acc, va[i], vb[i]);
    acc = warp_sum(acc);
    if (lane == 0) s_Y[a + BQ_NB * b] = sadd(acc, conjg(va[b]));
  }
  __syncthreads();
  // T(a, a) = tau_a, T(a, b) = -tau_b sum_{c=a}^{b-1} T(a, c) Y(c, b): each
  // row a is its own recurrence over b, one lane per row
  if (warp == 0 && lane < kmax) {
    const int a = lane;
    s_T[a + BQ_NB * a] = s_tau[a];
    for (int b = a + 1; b < kmax; ++b) {
      T acc = szero<T>();
      for (int c = a; c < b; ++c) mac(acc, s_T[a + BQ_NB * c], s_Y[c + BQ_NB * b]);
      s_T[a + BQ_NB * b] = smul(make_scalar<T>(-sreal(s_tau[b]), -simag(s_tau[b])), acc);
    }
  }
  __syncthreads();
  // rows p - off .. p - 1 (final after the previous panel's update), then
  // the panel: R on and above the diagonal, the v_k below
  for (int j = ec; j < kb; j += 16)
    for (int i = er - off; i < mp; i += 64) {
      T v = P[i + (size_t)ld * j];
      if (pexp != 0 && i >= 0 && i <= j) v = make_scalar<T>(scalbn(sreal(v), pexp), scalbn(simag(v), pexp));
      A[(size_t)(p + i) + (size_t)m * (p + j)] = v;
    }
  // V^T rows with the implicit unit diagonal and the zeros above it
  for (int a = ec; a < kb; a += 16)
    for (int i = er; i < mp; i += 64)
      Vt[i + (size_t)mp * a] = (i == a) ? sone(T()) : (i > a && a < kmax) ? P[i + (size_t)ld * a] : szero<T>();
  for (int e = tid; e < BQ_NB * BQ_NB; e += BQP_THREADS) Tm[e] = s_T[e];
}

// The CTA's columns cbase + [0, BQ_CB) that lie in [clo, chi), held in
// shared memory (sX: column c at sX + ldx c, global row g at index g - xr0),
// <- (I - V op(T) V^H) X[p:m, c] with V^T = Vt (kb rows of mp = m - p, ld
// mp).  adj = 1: op(T) = T^H (applies Q^H, the trailing update); adj = 0:
// op(T) = T (forms Q).  V is first staged in shared memory (sV: one
// contiguous copy of V^T, so every later read is a shared-memory read and
// the L2 latency is paid once), then W = V^H X by warps (AW reflectors x
// BQ_CB columns each, lanes over rows), op(T) W, and one warp per column for
// X -= V W'.  RG row groups (RG * 32 * BQ_CB threads): each warp covers every
// RG-th 32-row stripe and the RG partial sums of W are added in group order.
// A column's arithmetic does not depend on which other columns share the
// CTA (for a given RG).
template <typename T, int CB, int RG>
__device__ __forceinline__ void bq_apply_staged(T* __restrict__ sX, int ldx, int xr0, int cbase,
                                                int clo, int chi, const T* __restrict__ Vt, int m,
                                                int p, int kb, const T* __restrict__ Tm, int adj,
                                                T* __restrict__ sV, T (&W)[RG][BQ_NB][CB],
                                                T (&W2)[BQ_NB][CB]) {
  constexpr int NT = 32 * CB * RG;
  const int tid = threadIdx.x, lane = tid & 31;
  const int warp = (tid >> 5) % CB, rg = (tid >> 5) / CB;
  const int mp = m - p;
  for (int e = tid; e < mp * kb; e += NT) sV[e] = Vt[e];
  __syncthreads();
  constexpr int AW = BQ_NB / CB;   // reflectors per warp (CB warps x AW = BQ_NB)
  T acc[AW][CB];
#pragma unroll
  for (int u = 0; u < AW; ++u)
#pragma unroll
    for (int c = 0; c < CB; ++c) acc[u][c] = szero<T>();
  const T* xs = sX + (p - xr0);
  for (int i = 32 * rg + lane; i < mp; i += 32 * RG) {
    T x[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      const int col = cbase + c;
      x[c] = (col >= clo && col < chi) ? xs[i + ldx * c] : szero<T>();
    }
#pragma unroll
    for (int u = 0; u < AW; ++u) {
      const int a = warp * AW + u;
      const T v = (a < kb) ? sV[i + mp * a] : szero<T>();
#pragma unroll
      for (int c = 0; c < CB; ++c) macc(acc[u][c], v, x[c]);
    }
  }
#pragma unroll
  for (int u = 0; u < AW; ++u)
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      const T w = warp_sum(acc[u][c]);
      if (lane == 0) W[rg][warp * AW + u][c] = w;
    }
  __syncthreads();
  for (int e = tid; e < BQ_NB * CB; e += NT) {
    const int a = e % BQ_NB, c = e / BQ_NB;
    if (RG > 1) {   // the row groups' partials, in group order
      T w = W[0][a][c];
      for (int g = 1; g < RG; ++g) w = sadd(w, W[g][a][c]);
      W[0][a][c] = w;
    }
  }
  if (RG > 1) __syncthreads();
  for (int e = tid; e < BQ_NB * CB; e += NT) {
    const int a = e % BQ_NB, c = e / BQ_NB;
    T w2 = szero<T>();
    if (a < kb) {
      if (adj) {
        for (int b = 0; b <= a; ++b) macc(w2, Tm[b + BQ_NB * a], W[0][b][c]);   // conj(T[b, a])
      } else {
        for (int b = a; b < kb; ++b) mac(w2, Tm[a + BQ_NB * b], W[0][b][c]);
      }
    }
    W2[a][c] = w2;
  }
  __syncthreads();
  const int col = cbase + warp;
  if (col >= clo && col < chi) {
    T* xc = sX + (p - xr0) + (size_t)ldx * warp;
    for (int i = 32 * rg + lane; i < mp; i += 32 * RG) {
      T sacc = szero<T>();
      for (int a = 0; a < kb; ++a) mac(sacc, sV[i + mp * a], W2[a][warp]);
      xc[i] = ssub(xc[i], sacc);
    }
  }
  __syncthreads();   // sV and the updated columns are read again by the next use
}

// shared memory of the two kernels below: the CTA's columns (up to BQ_MAXM
// rows each) and one panel's V^T
constexpr size_t bq_apply_smem_elems() { return (size_t)BQ_MAXM * (BQ_CB + BQ_NB); }

// X[p:m, c] <- (I - V op(T) V^H) X[p:m, c] for the columns c of this CTA
// (col0 + BQ_CB blockIdx.x + [0, BQ_CB), below col0 + ncols): the columns
// are read into shared memory once (one warp per column), updated there
// and written back
template <typename T>
__global__ void __launch_bounds__(32 * BQ_CB)
k_bq_apply(T* __restrict__ X, int m, int col0, int ncols, const T* __restrict__ Vt, int p, int kb,
           const T* __restrict__ Tm, int adj) {
  extern __shared__ __align__(16) unsigned char bq_asmem[];
  __shared__ T W[1][BQ_NB][BQ_CB];
  __shared__ T W2[BQ_NB][BQ_CB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mp = m - p;
  T* sX = reinterpret_cast<T*>(bq_asmem);
  T* sV = sX + (size_t)mp * BQ_CB;
  const int cbase = col0 + BQ_CB * (int)blockIdx.x;
  const int col = cbase + warp;
  const bool mine = col < col0 + ncols;
  if (mine)
    for (int i = lane; i < mp; i += 32) sX[i + (size_t)mp * warp] = X[(size_t)(p + i) + (size_t)m * col];
  bq_apply_staged<T, BQ_CB, 1>(sX, mp, p, cbase, col0, col0 + ncols, Vt, m, p, kb, Tm, adj, sV, W, W2);
  if (mine)
    for (int i = lane; i < mp; i += 32) X[(size_t)(p + i) + (size_t)m * col] = sX[i + (size_t)mp * warp];
}

// Q formation in one launch: the CTA's columns cbase + [0, BQF_CB) of Q start
// as columns of the identity in shared memory and pass through the panels'
// block reflectors from the last panel to the first (panel pi touches the
// columns in [p, nq)), without a grid-wide step between panels (the columns
// are independent); then they are written to Q.  Each CTA streams every
// panel's V through its shared memory and updates only BQF_CB columns, so
// the work spreads over nq / BQF_CB SMs; BQF_RG row groups give each column
// several warps.
constexpr int BQF_CB = 2, BQF_RG = 4;
template <typename T>
__global__ void __launch_bounds__(32 * BQF_CB * BQF_RG)
k_bq_formq(T* __restrict__ Q, int m, int nq, int kmax, const T* __restrict__ Vall,
           const T* __restrict__ Tm) {
  extern __shared__ __align__(16) unsigned char bq_fsmem[];
  __shared__ T W[BQF_RG][BQ_NB][BQF_CB];
  __shared__ T W2[BQ_NB][BQF_CB];
  const int warp = (threadIdx.x >> 5) % BQF_CB, rg = (threadIdx.x >> 5) / BQF_CB;
  const int lane = threadIdx.x & 31;
  T* sX = reinterpret_cast<T*>(bq_fsmem);
  T* sV = sX + (size_t)m * BQF_CB;
  const int cbase = BQF_CB * (int)blockIdx.x;
  const int col = cbase + warp;
  for (int i = 32 * rg + lane; i < m; i += 32 * BQF_RG)
    sX[i + (size_t)m * warp] = (i == col) ? sone(T()) : szero<T>();
  __syncthreads();
  const int np = (kmax + BQ_NB - 1) / BQ_NB;
  for (int pi = np - 1; pi >= 0; --pi) {
    const int p = pi * BQ_NB;
    if (p >= nq || cbase + BQF_CB <= p) continue;   // block-uniform: no column of this CTA
    const int kb = min(BQ_NB, kmax - p);
    bq_apply_staged<T, BQF_CB, BQF_RG>(sX, m, 0, cbase, p, nq, Vall + (size_t)pi * BQ_NB * BQ_MAXM,
                                       m, p, kb, Tm + (size_t)pi * BQ_NB * BQ_NB, 0, sV, W, W2);
  }
  if (col < nq)
    for (int i = 32 * rg + lane; i < m; i += 32 * BQF_RG)
      Q[(size_t)i + (size_t)m * col] = sX[i + (size_t)m * warp];
}

// A[i + m j] = conj(S[j + ls i])  (A = S^H, m x n, from S n x m)
template <typename T>
__global__ void k_conj_transpose(const T* S, int ls, int n, int m, T* A) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)m * n) return;
  const int i = (int)(e % m), j = (int)(e / m);
  A[e] = conjg(S[j + (size_t)ls * i]);
}

// workspace of big_qr_q: T of every panel, then V^T of every panel
size_t big_qr_tm_elems(int n) {
  const size_t np = (size_t)((n + BQ_NB - 1) / BQ_NB);
  return np * BQ_NB * BQ_NB + np * BQ_NB * BQ_MAXM;
}

static std::atomic<unsigned long long> g_bq_cfg[2];

template <typename T>
static void bq_configure() {
  if (first_on_device(&g_bq_cfg[Sc<T>::cplx ? 0 : 1]))
  {
    cudaFuncSetAttribute(k_bq_panel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(T) * (BQ_MAXM + 1) * BQ_NB));
    cudaFuncSetAttribute(k_bq_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(T) * bq_apply_smem_elems()));
    cudaFuncSetAttribute(k_bq_formq<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(T) * bq_apply_smem_elems()));
  }
}

// per host thread and device: the side stream of the QR look-ahead and the
// two events that fork it from and join it to the caller's stream
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
static SideStream* side_stream() {
  thread_local SideStream tab[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  SideStream& e = tab[dev];
  if (!e.s) {
    if (cudaStreamCreateWithFlags(&e.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e.join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      e = SideStream();
      return nullptr;
    }
  }
  return &e;
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
  const int np = (kmax + BQ_NB - 1) / BQ_NB;
  T* Vall = Tm + (size_t)((n + BQ_NB - 1) / BQ_NB) * BQ_NB * BQ_NB;   // V^T of panel pi at pi NB MAXM
  // look-ahead: the kernel of panel p + NB first applies panel p's
  // reflectors to its own columns, so after panel p only the columns beyond
  // the next panel remain; they are updated on a side stream while the next
  // panel is factored.  Every column receives the same updates in the same
  // order (and the same arithmetic) as without the split.  The side stream
  // forks from s and joins it by events, so the sequence is also valid
  // inside a stream capture.
  SideStream* ss = side_stream();
  const bool ahead = ss && np > 2;
  if (ahead) {
    cudaEventRecord(ss->fork, s);
    cudaStreamWaitEvent(ss->s, ss->fork, 0);
  }
  bool join_pending = false;
  for (int p = 0; p < kmax; p += BQ_NB) {
    const int kb = std::min(BQ_NB, kmax - p);
    T* Tp = Tm + (size_t)(p / BQ_NB) * BQ_NB * BQ_NB;
    T* Vp = Vall + (size_t)(p / BQ_NB) * BQ_NB * BQ_MAXM;
    // algorithmic work (complex flop = 4 real multiplies + 4 adds): the
    // Householder factorisation of the (m - p) x kb panel, 8 kb^2 (M - kb/3),
    // and a block-reflector application to nc columns, 16 M kb nc
    const double M = (double)(m - p);
    const double cplx = Sc<T>::cplx ? 1.0 : 0.25;
    const bool fuse = ahead && p > 0;
    {
      QTT_PROF("bigqr_panel", s);
      prof_add_work("bigqr_panel", cplx * 8.0 * kb * kb * (M - kb / 3.0), 2.0 * M * kb * sizeof(T));
      if (fuse)
        prof_add_work("bigqr_panel", cplx * 16.0 * (M + BQ_NB) * BQ_NB * kb, 0.0);
      const T* Vprev = fuse ? Vp - (size_t)BQ_NB * BQ_MAXM : nullptr;
      const T* Tprev = fuse ? Tp - (size_t)BQ_NB * BQ_NB : nullptr;
      const int rows = (m - p) + (fuse ? BQ_NB : 0);
      const size_t smem = sizeof(T) * (size_t)(rows | 1) * kb;
      k_bq_panel<T, 1><<<1, BQP_THREADS, smem, s>>>(A, m, p, kb, Tp, Vp, Vprev, Tprev, BQ_NB);
    }
    const int c0 = p + kb, nc = kmax - c0;
    const size_t asmem = sizeof(T) * (size_t)(m - p) * (BQ_CB + kb);
    if (ahead) {
      // the next panel needs the side stream's update from the panel before
      if (join_pending) {
        cudaStreamWaitEvent(s, ss->join, 0);
        join_pending = false;
      }
      const int nn = std::min(BQ_NB, std::max(nc, 0));
      if (nc > nn) {
        cudaEventRecord(ss->fork, s);                 // panel p done
        cudaStreamWaitEvent(ss->s, ss->fork, 0);
        prof_add_work("bigqr_update", cplx * 16.0 * M * kb * (nc - nn), 2.0 * M * (nc - nn) * sizeof(T));
        k_bq_apply<T><<<(nc - nn + BQ_CB - 1) / BQ_CB, 32 * BQ_CB, asmem, ss->s>>>(
            A, m, c0 + nn, nc - nn, Vp, p, kb, Tp, 1);
        cudaEventRecord(ss->join, ss->s);
        join_pending = true;
      }
    } else if (nc > 0) {
      QTT_PROF("bigqr_update", s);
      prof_add_work("bigqr_update", cplx * 16.0 * M * kb * nc, 2.0 * M * nc * sizeof(T));
      k_bq_apply<T><<<(nc + BQ_CB - 1) / BQ_CB, 32 * BQ_CB, asmem, s>>>(A, m, c0, nc, Vp, p, kb, Tp, 1);
    }
  }
  if (ahead) {
    cudaEventRecord(ss->join, ss->s);   // the side stream's last work joins s
    cudaStreamWaitEvent(s, ss->join, 0);
  }
  {
    QTT_PROF("bigqr_formq", s);
    for (int pi = np - 1; pi >= 0; --pi) {
      const int p = pi * BQ_NB;
      const int kb = std::min(BQ_NB, kmax - p);
      if (p >= nq) continue;
      prof_add_work("bigqr_formq", (Sc<T>::cplx ? 1.0 : 0.25) * 16.0 * (m - p) * kb * (double)(nq - p),
                    2.0 * (m - p) * (double)(nq - p) * sizeof(T));
    }
    k_bq_formq<T><<<(nq + BQF_CB - 1) / BQF_CB, 32 * BQF_CB * BQF_RG,
                    sizeof(T) * (size_t)m * (BQF_CB + BQ_NB), s>>>(Q, m, nq, kmax, Vall, Tm);
  }
  return cuda_check(cudaGetLastError(), "big_qr launch");
}
template qtt_status big_qr_q<float2>(float2*, int, int, int, float2*, float2*, cudaStream_t);
template qtt_status big_qr_q<double>(double*, int, int, int, double*, double*, cudaStream_t);

template <typename T>
static qtt_status debug_big_qr(const void* A, int m, int n, int nq, void* Q, cudaStream_t s) {
  T* Aw = (T*)scratch_alloc(sizeof(T) * (size_t)m * n, s);
  T* Tm = (T*)scratch_alloc(sizeof(T) * big_qr_tm_elems(n), s);
  qtt_status st = QTT_ENOMEM;
  if (Aw && Tm) {
    st = cuda_check(cudaMemcpyAsync(Aw, A, sizeof(T) * (size_t)m * n, cudaMemcpyDeviceToDevice, s),
                    "big_qr copy");
    if (st == QTT_OK) st = big_qr_q<T>(Aw, m, n, nq, (T*)Q, Tm, s);
  } else {
    set_error("qtt_debug_big_qr: scratch allocation failed");
  }
  if (Aw) scratch_free(Aw, s);
  if (Tm) scratch_free(Tm, s);
  return st;
}

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

// One 64 x 64 output tile of batch z % nbatch over the k range of split
// z / nbatch (kchunk terms each).  The next k chunk's operands are loaded
// into registers while the current one is multiplied from shared memory
// (two buffers, one barrier per chunk).  With splits > 1 the tile's partial
// sum goes to part + split * ldpart (ld M), summed by k_cgemm_reduce.
template <typename TA>
__global__ void __launch_bounds__(CG_THREADS, 1)
k_cgemm(CGemmArgs<TA> g, int nbatch, int kchunk, float2* __restrict__ part, long long ldpart) {
  __shared__ TA As[2][CG_BK][CG_BM + 1];
  __shared__ float2 Bs[2][CG_BK][CG_BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int bz = blockIdx.z % nbatch, split = blockIdx.z / nbatch;
  const int b1 = bz % g.nb1, b2 = bz / g.nb1;
  const TA* A = g.A + g.bA1 * b1 + g.bA2 * b2;
  const float2* B = g.B + g.bB1 * b1 + g.bB2 * b2;
  const long long i0 = (long long)blockIdx.y * CG_BM, j0 = (long long)blockIdx.x * CG_BN;
  const int kbeg = split * kchunk;
  const int kend = min(g.K, kbeg + kchunk);
  const bool a_rows_unit = (g.sAi == 1);
  float2 sum[4][4], cmp[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      sum[u][v] = make_float2(0.f, 0.f);
      cmp[u][v] = make_float2(0.f, 0.f);
    }
  constexpr int LA = CG_BM * CG_BK / CG_THREADS;   // 4 elements of A and of B per thread
  TA ra[LA];
  float2 rb[LA];
  auto load = [&](int k0) {
#pragma unroll
    for (int t = 0; t < LA; ++t) {
      const int e = tid + CG_THREADS * t;
      int ii, kk;
      if (a_rows_unit) { ii = e % CG_BM; kk = e / CG_BM; }
      else { kk = e % CG_BK; ii = e / CG_BK; }
      const long long i = i0 + ii;
      const int k = k0 + kk;
      TA v = cg_zero(TA());
      if (i < g.M && k < kend) {
        v = A[i * g.sAi + (long long)k * g.sAk];
        if (g.conjA) v = cg_conj(v);
      }
      ra[t] = v;
      const int kb = e % CG_BK, jj = e / CG_BK;
      const long long j = j0 + jj;
      const int k2 = k0 + kb;
      rb[t] = (j < g.N && k2 < kend) ? B[(long long)k2 * g.sBk + j * g.sBj] : make_float2(0.f, 0.f);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int t = 0; t < LA; ++t) {
      const int e = tid + CG_THREADS * t;
      int ii, kk;
      if (a_rows_unit) { ii = e % CG_BM; kk = e / CG_BM; }
      else { kk = e % CG_BK; ii = e / CG_BK; }
      As[buf][kk][ii] = ra[t];
      Bs[buf][e % CG_BK][e / CG_BK] = rb[t];
    }
  };
  if (kbeg < kend) {
    load(kbeg);
    store(0);
  }
  __syncthreads();
  int buf = 0;
  for (int k0 = kbeg; k0 < kend; k0 += CG_BK) {
    const bool more = k0 + CG_BK < kend;
    if (more) load(k0 + CG_BK);
    float2 pt[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) pt[u][v] = make_float2(0.f, 0.f);
#pragma unroll
    for (int kk = 0; kk < CG_BK; ++kk) {
      TA a[4];
      float2 b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[buf][kk][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Bs[buf][kk][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) cg_mac(pt[u][v], a[u], b[v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) cg_kadd(sum[u][v], cmp[u][v], pt[u][v]);
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  float2* C = part ? part + (long long)split * ldpart : g.C + g.bC1 * b1 + g.bC2 * b2;
  const long long sCi = part ? 1 : g.sCi, sCj = part ? g.M : g.sCj;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const long long i = i0 + ty + 16 * u;
    if (i >= g.M) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const long long j = j0 + tx + 16 * v;
      if (j >= g.N) continue;
      C[i * sCi + j * sCj] = make_float2(sum[u][v].x - cmp[u][v].x, sum[u][v].y - cmp[u][v].y);
    }
  }
}

// C[i, j] = sum over splits of part[s][i + M j], compensated, in split order
__global__ void k_cgemm_reduce(const float2* __restrict__ part, int splits, long long ldpart, int M,
                               int N, float2* __restrict__ C, long long sCi, long long sCj) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)M * N) return;
  const long long i = e % M, j = e / M;
  float2 sm = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
  for (int s2 = 0; s2 < splits; ++s2) cg_kadd(sm, c, part[e + (long long)s2 * ldpart]);
  C[i * sCi + j * sCj] = make_float2(sm.x - c.x, sm.y - c.y);
}

void cgemm_reduce(const float2* part, int splits, long long ldpart, int M, int N, float2* C,
                  long long sCi, long long sCj, cudaStream_t s) {
  k_cgemm_reduce<<<(unsigned)((ldpart + 255) / 256), 256, 0, s>>>(part, splits, ldpart, M, N, C, sCi,
                                                                  sCj);
}

template <typename TA>
qtt_status cgemm(const CGemmArgs<TA>& g, int nbatch, cudaStream_t s, const char* name) {
  if (g.M <= 0 || g.N <= 0 || nbatch <= 0) return QTT_OK;
  if (g.nb1 < 1 || nbatch > 65535) {
    set_error("cgemm: bad batch (%d, nb1 %d)", nbatch, g.nb1);
    return QTT_EINVAL;
  }
  if ((g.M + CG_BM - 1) / CG_BM > 65535) {
    set_error("cgemm: M = %d too large", g.M);
    return QTT_EINVAL;
  }
  const long long tiles = (long long)((g.N + CG_BN - 1) / CG_BN) * ((g.M + CG_BM - 1) / CG_BM);
  // split k when the tiles alone cannot fill the GPU (one batch, long k)
  const int sms = device_sm_count();
  int splits = 1;
  if (nbatch == 1 && tiles < 2LL * sms && g.K >= 8 * CG_BK) {
    splits = (int)std::min<long long>((2LL * sms + tiles - 1) / tiles, (long long)g.K / (4 * CG_BK));
    splits = std::max(1, std::min(splits, 16));
  }
  const int kchunk = ((g.K + splits - 1) / splits + CG_BK - 1) / CG_BK * CG_BK;
  dim3 grid((unsigned)((g.N + CG_BN - 1) / CG_BN), (unsigned)((g.M + CG_BM - 1) / CG_BM),
            (unsigned)(nbatch * splits));
  QTT_PROF(name, s);
  const double mnk = (double)g.M * g.N * g.K * nbatch;
  prof_add_work(name, (sizeof(TA) == sizeof(float) ? 4.0 : 8.0) * mnk,
                ((double)g.M * g.K * sizeof(TA) + (double)g.K * g.N * 8.0 + (double)g.M * g.N * 8.0) *
                    nbatch);
  if (splits == 1) {
    k_cgemm<TA><<<grid, CG_THREADS, 0, s>>>(g, nbatch, kchunk, nullptr, 0);
    return QTT_OK;
  }
  const long long ldpart = (long long)g.M * g.N;
  float2* part = (float2*)scratch_alloc(sizeof(float2) * (size_t)(ldpart * splits), s);
  if (!part) {
    set_error("cgemm: split-k scratch allocation failed");
    return QTT_ENOMEM;
  }
  k_cgemm<TA><<<grid, CG_THREADS, 0, s>>>(g, 1, kchunk, part, ldpart);
  cgemm_reduce(part, splits, ldpart, g.M, g.N, g.C, g.sCi, g.sCj, s);
  scratch_free(part, s);
  return QTT_OK;
}

template qtt_status cgemm<float>(const CGemmArgs<float>&, int, cudaStream_t, const char*);
template qtt_status cgemm<float2>(const CGemmArgs<float2>&, int, cudaStream_t, const char*);

}  // namespace qtt

extern "C" qtt_status qtt_debug_big_qr(const void* A, int m, int n, int nq, int dtype, void* Q,
                                      void* stream) {
  qtt::clear_error();
  if (!A || !Q || m < 1 || n < 1 || nq < 1 || nq > m || m > 1024 ||
      (dtype != QTT_C64 && dtype != QTT_F64)) {
    qtt::set_error("qtt_debug_big_qr: NULL array, shape %d x %d (nq %d) or dtype %d not accepted",
                   m, n, nq, dtype);
    return QTT_EINVAL;
  }
  const cudaStream_t s = (cudaStream_t)stream;
  return dtype == QTT_C64 ? qtt::debug_big_qr<float2>(A, m, n, nq, Q, s)
                          : qtt::debug_big_qr<double>(A, m, n, nq, Q, s);
}
