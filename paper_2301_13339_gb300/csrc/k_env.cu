// Differentiation of the convolution step: environment sweeps, TT sums and
// the adjoint operator.
//
//  * Inner product <x, y> = sum_n conj(x[n]) y[n] of two QTT tensors by a
//    left-to-right sweep of the environments
//        E_k = sum_{a, i} conj(X_k[a, i, :])^T E_{k-1}[a, :] Y_k[:, i, :]
//    (E_0 = 1, E_d = <x, y>).
//  * Core gradients of f -> ||T full(f) - g||^2 (chain rule through Full,
//    Alg. 3): for a QTT vector w,
//        grad_k[a, i, b] = sum_{a', b'} E_{k-1}[a, a'] W_k[a', i, b'] R_k[b', b]
//    with the left environments E of (f, w) and the right environments R
//    built in a right-to-left sweep.  With w = 2 T^H (T f - g) this is
//    2 dL/d conj(F_k) (the gradient PyTorch uses for complex leaves).
//  * TT sum alpha x + beta y (block-diagonal cores, ranks add).
//  * Transposed operator cores (T^H for the real operator cores of the sinc
//    Toeplitz matrix: O_k[p, j, i, q] -> O_k[p, i, j, q]).
//
// All sweeps run in one CTA: the environments are at most 64 x 64 and the
// d-step chain is sequential, so the cost is the latency of d small
// contractions held in shared memory.
#include "qtt_internal.cuh"
#include <algorithm>
#include <type_traits>

namespace qtt {

namespace {

constexpr int ENV_THREADS = 512;
constexpr int ENV_MAXD = 32;

template <typename T>
struct EnvArgs {
  const T* F;
  const T* W;
  size_t foff[ENV_MAXD];
  size_t woff[ENV_MAXD];
  T* grad[ENV_MAXD];
  const int* fr;
  const int* wr;
  int d;
  T* Est;          // stored left environments, slot k (k = 0..d-1) at k*ecap
  int ecap;        // max_k rfcap_k * rwcap_k
  double alpha;    // grad_k = alpha * (E W R) + beta * grad_k
  double beta;
  double2* dot_out;
  int want_grads;
};

__device__ __forceinline__ double one_of(double) { return 1.0; }
__device__ __forceinline__ float2 one_of(float2) { return make_float2(1.f, 0.f); }

// Z[a + r0f (i + 2 b')] = sum_{a'} E[a + r0f a'] W[a' + r0w (i + 2 b')]
template <typename T>
__device__ void env_times_core(const T* E, const T* __restrict__ Wk, int r0f, int r0w, int r1w,
                               T* Z) {
  const int n = r0f * 2 * r1w;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int a = e % r0f, c = e / r0f;
    const T* wc = Wk + (size_t)r0w * c;
    T acc = szero<T>();
    for (int ap = 0; ap < r0w; ++ap) mac(acc, E[a + r0f * ap], __ldg(wc + ap));
    Z[e] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(ENV_THREADS) env_sweep_kernel(EnvArgs<T> A) {
  extern __shared__ __align__(16) unsigned char env_smem[];
  T* E = (T*)env_smem;
  T* X = E + A.ecap;
  T* Rm = X + 2 * (size_t)A.ecap;
  const int d = A.d;
  if (threadIdx.x == 0) {
    E[0] = one_of(T());
    if (A.want_grads) A.Est[0] = E[0];
  }
  __syncthreads();
  // ---- left sweep
  for (int k = 1; k <= d; ++k) {
    const int r0f = A.fr[k - 1], r1f = A.fr[k], r0w = A.wr[k - 1], r1w = A.wr[k];
    const T* Fk = A.F + A.foff[k - 1];
    const T* Wk = A.W + A.woff[k - 1];
    env_times_core(E, Wk, r0f, r0w, r1w, X);
    __syncthreads();
    const int n = r1f * r1w;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int b = e % r1f, bp = e / r1f;
      T acc = szero<T>();
      for (int i = 0; i < 2; ++i) {
        const T* fc = Fk + (size_t)r0f * (i + 2 * b);
        const T* zc = X + (size_t)r0f * (i + 2 * bp);
        for (int a = 0; a < r0f; ++a) macc(acc, __ldg(fc + a), zc[a]);
      }
      E[e] = acc;
      if (A.want_grads && k < d) A.Est[(size_t)k * A.ecap + e] = acc;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && A.dot_out) *A.dot_out = to_d2(E[0]);
  if (!A.want_grads) return;
  __syncthreads();
  // ---- right sweep with the gradients
  if (threadIdx.x == 0) Rm[0] = one_of(T());
  for (int k = d; k >= 1; --k) {
    const int r0f = A.fr[k - 1], r1f = A.fr[k], r0w = A.wr[k - 1], r1w = A.wr[k];
    const T* Fk = A.F + A.foff[k - 1];
    const T* Wk = A.W + A.woff[k - 1];
    for (int e = threadIdx.x; e < r0f * r0w; e += blockDim.x)
      E[e] = A.Est[(size_t)(k - 1) * A.ecap + e];
    __syncthreads();
    env_times_core(E, Wk, r0f, r0w, r1w, X);
    __syncthreads();
    // grad_k[a + r0f (i + 2 b)] = alpha sum_{b'} Z[a + r0f (i + 2 b')] Rm[b' + r1w b]
    T* G = A.grad[k - 1];
    const int ng = r0f * 2 * r1f;
    for (int e = threadIdx.x; e < ng; e += blockDim.x) {
      const int a = e % r0f, i = (e / r0f) % 2, b = e / (2 * r0f);
      T acc = szero<T>();
      for (int bp = 0; bp < r1w; ++bp) mac(acc, X[a + r0f * (i + 2 * bp)], Rm[bp + r1w * b]);
      T v = rscale(acc, (typename Sc<T>::R)A.alpha);
      if (A.beta != 0.0) v = sadd(v, rscale(G[e], (typename Sc<T>::R)A.beta));
      G[e] = v;
    }
    __syncthreads();
    if (k == 1) break;
    // V[b' + r1w (a + r0f i)] = sum_b Rm[b' + r1w b] conj(F_k[a + r0f (i + 2 b)])
    const int nv = r1w * r0f * 2;
    for (int e = threadIdx.x; e < nv; e += blockDim.x) {
      const int bp = e % r1w, a = (e / r1w) % r0f, i = e / (r1w * r0f);
      T acc = szero<T>();
      for (int b = 0; b < r1f; ++b) macb(acc, Rm[bp + r1w * b], __ldg(Fk + a + (size_t)r0f * (i + 2 * b)));
      X[e] = acc;
    }
    __syncthreads();
    // Rm_new[a' + r0w a] = sum_{i, b'} W_k[a' + r0w (i + 2 b')] V[b' + r1w (a + r0f i)]
    const int nr = r0w * r0f;
    for (int e = threadIdx.x; e < nr; e += blockDim.x) {
      const int ap = e % r0w, a = e / r0w;
      T acc = szero<T>();
      for (int i = 0; i < 2; ++i)
        for (int bp = 0; bp < r1w; ++bp)
          mac(acc, __ldg(Wk + ap + (size_t)r0w * (i + 2 * bp)), X[bp + r1w * (a + r0f * i)]);
      Rm[e] = acc;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- TT sum
// out_k = [alpha X_1, beta Y_1] (k = 1), diag(X_k, Y_k) (1 < k < d),
// [X_d; Y_d] (k = d); ranks rx + ry in the interior.
template <typename T>
__global__ void tt_add_core_kernel(const T* __restrict__ X, const int* __restrict__ xr,
                                   const T* __restrict__ Y, const int* __restrict__ yr, int k, int d,
                                   double alpha, double beta, T* __restrict__ Z, int* __restrict__ zr,
                                   long long capel) {
  const int x0 = xr[k - 1], x1 = xr[k], y0 = yr[k - 1], y1 = yr[k];
  const int R0 = (k == 1) ? 1 : x0 + y0;
  const int R1 = (k == d) ? 1 : x1 + y1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    zr[k] = R1;
    if (k == 1) zr[0] = 1;
  }
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)R0 * 2 * R1 || e >= capel) return;
  const int a = (int)(e % R0), i = (int)((e / R0) % 2), b = (int)(e / (2LL * R0));
  T v = szero<T>();
  if (k == 1) {
    if (b < x1) v = rscale(X[(size_t)(i + 2 * b)], (typename Sc<T>::R)alpha);
    else v = rscale(Y[(size_t)(i + 2 * (b - x1))], (typename Sc<T>::R)beta);
  } else if (k == d) {
    if (a < x0) v = X[a + (size_t)x0 * i];
    else v = Y[(a - x0) + (size_t)y0 * i];
  } else {
    if (a < x0 && b < x1) v = X[a + (size_t)x0 * (i + 2 * b)];
    else if (a >= x0 && b >= x1) v = Y[(a - x0) + (size_t)y0 * (i + 2 * (b - x1))];
  }
  Z[e] = v;
}

// ---------------------------------------------------------------- transpose
template <typename R>
__global__ void op_transpose_kernel(const R* __restrict__ in, R* __restrict__ out, int P0, int P1) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= P0 * 4 * P1) return;
  const int p = e % P0, j = (e / P0) % 2, i = (e / (2 * P0)) % 2, q = e / (4 * P0);
  out[e] = in[p + P0 * (i + 2 * (j + 2 * q))];
}

// core k of t copied to its capacities c0 x 2 x c1 (zeros beyond the device ranks)
__global__ void k_env_pad(const float2* __restrict__ X, const int* __restrict__ xr, int k, int c0,
                          int c1, float2* __restrict__ Xp) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)c0 * 2 * c1) return;
  const int a = (int)(e % c0);
  const long long t = e / c0;
  const int i = (int)(t % 2), b = (int)(t / 2);
  const int r0 = xr[k - 1], r1 = xr[k];
  Xp[e] = (a < r0 && b < r1) ? X[a + (size_t)r0 * (i + 2 * b)] : make_float2(0.f, 0.f);
}

// grad_k (f's layout at its device ranks) = alpha Gp + beta grad_k, Gp at the capacities
__global__ void k_env_grad_out(const float2* __restrict__ Gp, const int* __restrict__ fr, int k,
                               int c0, int c1, double alpha, double beta, float2* __restrict__ G) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r0 = fr[k - 1], r1 = fr[k];
  if (e >= (long long)r0 * 2 * r1) return;
  const int a = (int)(e % r0);
  const long long t = e / r0;
  const int i = (int)(t % 2), b = (int)(t / 2);
  (void)c1;
  const float2 v = Gp[a + (size_t)c0 * (i + 2 * b)];
  float2 o = make_float2((float)alpha * v.x, (float)alpha * v.y);
  if (beta != 0.0) {
    o.x += (float)beta * G[e].x;
    o.y += (float)beta * G[e].y;
  }
  G[e] = o;
}

__global__ void k_env_one(float2* e) {
  if (threadIdx.x == 0) *e = make_float2(1.f, 0.f);
}
__global__ void k_env_dot_out(const float2* e, double2* out) {
  if (threadIdx.x == 0) *out = make_double2((double)e->x, (double)e->y);
}

// The sweeps of env_sweep_kernel for environments too large for one CTA's
// shared memory (the adjoint's ranks in the large-rank rounding mode): the
// same contractions as strided batched complex GEMMs (compensated chunk
// sums) over f and w zero-padded to their host rank capacities, the left
// environments stored per cut in global memory.
//   left:   X = E_{k-1} W_k;  E_k = F_k^H X  (F_k, X as (2 r0f) x r1 matrices)
//   right:  X = E_{k-1} W_k;  grad_k = alpha X R_k + beta grad_k;
//           Y_i = W_k[:, i, :] R_k;  R_{k-1}^T = conj(F_k) Y^T over (i, b)
static qtt_status env_sweep_big(const qtt_tensor* f, const qtt_tensor* w, double alpha, double beta,
                                void* const* grad, double2* dot_out, cudaStream_t s) {
  const int d = f->desc.d;
  const std::vector<int>& cf = f->rcap;
  const std::vector<int>& cw = w->rcap;
  size_t nf = 0, nw = 0, ne = 0, xmax = 1, rmax = 1, ymax = 1, gmax = 1;
  std::vector<size_t> fo(d), wo(d), eo(d + 1);
  for (int k = 1; k <= d; ++k) {
    fo[k - 1] = nf; nf += (size_t)cf[k - 1] * 2 * cf[k];
    wo[k - 1] = nw; nw += (size_t)cw[k - 1] * 2 * cw[k];
    xmax = std::max(xmax, (size_t)cf[k - 1] * 2 * cw[k]);
    rmax = std::max(rmax, (size_t)cw[k] * cf[k]);
    ymax = std::max(ymax, (size_t)cw[k - 1] * 2 * cf[k]);
    gmax = std::max(gmax, (size_t)cf[k - 1] * 2 * cf[k]);
  }
  for (int k = 0; k <= d; ++k) { eo[k] = ne; ne += (size_t)cf[k] * cw[k]; }
  const size_t tot = nf + nw + ne + 2 * xmax + 2 * rmax + ymax + gmax;
  float2* buf = (float2*)scratch_alloc(sizeof(float2) * tot, s);
  if (!buf) { set_error("environment sweep (large ranks): scratch"); return QTT_ENOMEM; }
  float2* Fp = buf;
  float2* Wp = Fp + nf;
  float2* Est = Wp + nw;
  float2* X = Est + ne;
  float2* R0 = X + 2 * xmax;
  float2* R1 = R0 + rmax;
  float2* Y = R1 + rmax;
  float2* Gp = Y + ymax;
  qtt_status st = QTT_OK;
  for (int k = 1; k <= d; ++k) {
    const long long n1 = (long long)cf[k - 1] * 2 * cf[k], n2 = (long long)cw[k - 1] * 2 * cw[k];
    QTT_PROF("env_pad", s);
    k_env_pad<<<(unsigned)((n1 + 255) / 256), 256, 0, s>>>((const float2*)f->cores + f->off[k - 1],
                                                          f->ranks, k, cf[k - 1], cf[k], Fp + fo[k - 1]);
    k_env_pad<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>((const float2*)w->cores + w->off[k - 1],
                                                          w->ranks, k, cw[k - 1], cw[k], Wp + wo[k - 1]);
  }
  k_env_one<<<1, 32, 0, s>>>(Est + eo[0]);
  // X (c0f x 2 c1w) = E (c0f x c0w) W_k (c0w x 2 c1w)
  auto times_core = [&](int k, const float2* E) {
    CGemmArgs<float2> g;
    g.A = E; g.sAi = 1; g.sAk = cf[k - 1];
    g.B = Wp + wo[k - 1]; g.sBk = 1; g.sBj = cw[k - 1];
    g.C = X; g.sCi = 1; g.sCj = cf[k - 1];
    g.M = cf[k - 1]; g.N = 2 * cw[k]; g.K = cw[k - 1];
    return cgemm<float2>(g, 1, s, "env_gemm");
  };
  for (int k = 1; k <= d && st == QTT_OK; ++k) {
    st = times_core(k, Est + eo[k - 1]);
    if (st != QTT_OK) break;
    CGemmArgs<float2> g;   // E_k (c1f x c1w) = F_k^H X, K = (a, i) over 2 c0f
    g.A = Fp + fo[k - 1]; g.sAi = 2LL * cf[k - 1]; g.sAk = 1; g.conjA = 1;
    g.B = X; g.sBk = 1; g.sBj = 2LL * cf[k - 1];
    g.C = Est + eo[k]; g.sCi = 1; g.sCj = cf[k];
    g.M = cf[k]; g.N = cw[k]; g.K = 2 * cf[k - 1];
    st = cgemm<float2>(g, 1, s, "env_gemm");
  }
  if (st == QTT_OK && dot_out) k_env_dot_out<<<1, 32, 0, s>>>(Est + eo[d], dot_out);
  if (st == QTT_OK && grad) {
    float2* Rm = R0;
    float2* Rn = R1;
    k_env_one<<<1, 32, 0, s>>>(Rm);
    for (int k = d; k >= 1 && st == QTT_OK; --k) {
      st = times_core(k, Est + eo[k - 1]);
      if (st != QTT_OK) break;
      {
        CGemmArgs<float2> g;   // Gp (2 c0f x c1f) = X (2 c0f x c1w) R_k (c1w x c1f)
        g.A = X; g.sAi = 1; g.sAk = 2LL * cf[k - 1];
        g.B = Rm; g.sBk = 1; g.sBj = cw[k];
        g.C = Gp; g.sCi = 1; g.sCj = 2LL * cf[k - 1];
        g.M = 2 * cf[k - 1]; g.N = cf[k]; g.K = cw[k];
        st = cgemm<float2>(g, 1, s, "env_gemm");
      }
      if (st != QTT_OK) break;
      {
        const long long ng = (long long)cf[k - 1] * 2 * cf[k];
        QTT_PROF("env_grad_out", s);
        k_env_grad_out<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(Gp, f->ranks, k, cf[k - 1], cf[k],
                                                                   alpha, beta, (float2*)grad[k - 1]);
      }
      if (k == 1) break;
      {
        CGemmArgs<float2> g;   // Y[a' + c0w (i + 2 b)] = sum_b' W[a' + c0w (i + 2 b')] R[b' + c1w b]
        g.A = Wp + wo[k - 1]; g.sAi = 1; g.sAk = 2LL * cw[k - 1]; g.bA1 = cw[k - 1];
        g.B = Rm; g.sBk = 1; g.sBj = cw[k];
        g.C = Y; g.sCi = 1; g.sCj = 2LL * cw[k - 1]; g.bC1 = cw[k - 1];
        g.M = cw[k - 1]; g.N = cf[k]; g.K = cw[k]; g.nb1 = 2;
        st = cgemm<float2>(g, 2, s, "env_gemm");
      }
      if (st != QTT_OK) break;
      {
        CGemmArgs<float2> g;   // R_{k-1}[a' + c0w a] = sum_{i, b} Y[a', i, b] conj(F[a, i, b])
        g.A = Fp + fo[k - 1]; g.sAi = 1; g.sAk = cf[k - 1]; g.conjA = 1;
        g.B = Y; g.sBk = cw[k - 1]; g.sBj = 1;
        g.C = Rn; g.sCi = cw[k - 1]; g.sCj = 1;
        g.M = cf[k - 1]; g.N = cw[k - 1]; g.K = 2 * cf[k];
        st = cgemm<float2>(g, 1, s, "env_gemm");
      }
      std::swap(Rm, Rn);
    }
  }
  scratch_free(buf, s);
  if (st != QTT_OK) return st;
  return cuda_check(cudaGetLastError(), "environment sweep (large ranks)");
}

}  // namespace

// diagnostics: 1 sends every complex64 sweep through the GEMM path
static int g_env_big = 0;
void set_env_big(int on) { g_env_big = (on != 0); }

size_t env_smem_bytes(const qtt_tensor* f, const qtt_tensor* w) {
  int fm = 1, wm = 1;
  for (int v : f->rcap) fm = std::max(fm, v);
  for (int v : w->rcap) wm = std::max(wm, v);
  return 4 * (size_t)fm * wm * elem_size(f->desc.dt);
}

template <typename T>
static qtt_status env_sweep_t(const qtt_tensor* f, const qtt_tensor* w, double alpha, double beta,
                              void* const* grad, double2* dot_out, cudaStream_t s) {
  const int d = f->desc.d;
  EnvArgs<T> A{};
  A.F = (const T*)f->cores;
  A.W = (const T*)w->cores;
  for (int k = 0; k < d; ++k) {
    A.foff[k] = f->off[k];
    A.woff[k] = w->off[k];
    A.grad[k] = grad ? (T*)grad[k] : nullptr;
  }
  A.fr = f->ranks;
  A.wr = w->ranks;
  A.d = d;
  int fm = 1, wm = 1;
  for (int v : f->rcap) fm = std::max(fm, v);
  for (int v : w->rcap) wm = std::max(wm, v);
  A.ecap = fm * wm;
  A.alpha = alpha;
  A.beta = beta;
  A.dot_out = dot_out;
  A.want_grads = grad ? 1 : 0;
  const size_t smem = 4 * (size_t)A.ecap * sizeof(T);
  if (smem > 227 * 1024 || (g_env_big && std::is_same<T, float2>::value)) {
    if constexpr (std::is_same<T, float2>::value)
      return env_sweep_big(f, w, alpha, beta, grad, dot_out, s);
    set_error("environment sweep: rank capacities %d x %d need %zu bytes of shared memory", fm, wm, smem);
    return QTT_EUNSUPPORTED;
  }
  A.Est = nullptr;
  if (grad) {
    A.Est = (T*)scratch_alloc(sizeof(T) * (size_t)d * A.ecap, s);
    if (!A.Est) { set_error("environment sweep: scratch"); return QTT_ENOMEM; }
  }
  static std::atomic<unsigned long long> cfg{0};
  if (first_on_device(&cfg))
    cudaFuncSetAttribute(env_sweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  {
    QTT_PROF(grad ? "env_grads" : "env_dot", s);
    env_sweep_kernel<T><<<1, ENV_THREADS, smem, s>>>(A);
  }
  qtt_status st = cuda_check(cudaGetLastError(), "environment sweep");
  if (A.Est) scratch_free(A.Est, s);
  return st;
}

qtt_status env_sweep(const qtt_tensor* f, const qtt_tensor* w, double alpha, double beta,
                     void* const* grad, double2* dot_out, cudaStream_t s) {
  if (f->desc.d != w->desc.d || f->desc.dt != w->desc.dt) {
    set_error("environment sweep: tensors differ in d or element type");
    return QTT_EINVAL;
  }
  if (f->desc.d > ENV_MAXD) { set_error("environment sweep: d above %d", ENV_MAXD); return QTT_EINVAL; }
  if (f->desc.dt == QTT_F64) return env_sweep_t<double>(f, w, alpha, beta, grad, dot_out, s);
  return env_sweep_t<float2>(f, w, alpha, beta, grad, dot_out, s);
}

qtt_status tt_add(double alpha, const qtt_tensor* x, double beta, const qtt_tensor* y,
                  cudaStream_t s, qtt_tensor** out) {
  const int d = x->desc.d;
  if (y->desc.d != d || y->desc.dt != x->desc.dt) {
    set_error("qtt_add: tensors differ in d or element type");
    return QTT_EINVAL;
  }
  std::vector<int> cap(d + 1, 1);
  for (int k = 1; k < d; ++k) {
    cap[k] = x->rcap[k] + y->rcap[k];
    if (cap[k] > QTT_PRODUCT_CAP) { set_error("qtt_add: rank capacity above %d", QTT_PRODUCT_CAP); return QTT_EINVAL; }
  }
  qtt_tensor* z = nullptr;
  qtt_status st = tensor_alloc(x->desc, cap, s, &z);
  if (st != QTT_OK) return st;
  for (int k = 1; k <= d; ++k) {
    const long long capel = (long long)cap[k - 1] * 2 * cap[k];
    const unsigned blocks = (unsigned)((capel + 255) / 256);
    QTT_PROF("tt_add", s);
    if (x->desc.dt == QTT_F64)
      tt_add_core_kernel<double><<<blocks, 256, 0, s>>>(
          (const double*)x->cores + x->off[k - 1], x->ranks, (const double*)y->cores + y->off[k - 1],
          y->ranks, k, d, alpha, beta, (double*)z->cores + z->off[k - 1], z->ranks, capel);
    else
      tt_add_core_kernel<float2><<<blocks, 256, 0, s>>>(
          (const float2*)x->cores + x->off[k - 1], x->ranks, (const float2*)y->cores + y->off[k - 1],
          y->ranks, k, d, alpha, beta, (float2*)z->cores + z->off[k - 1], z->ranks, capel);
  }
  st = cuda_check(cudaGetLastError(), "qtt_add");
  if (st != QTT_OK) { tensor_free_async(z, s); return st; }
  *out = z;
  return QTT_OK;
}

qtt_status op_transpose(const qtt_op* op, cudaStream_t s, qtt_op** out) {
  qtt_op* t = new qtt_op();
  t->d = op->d;
  t->dt = op->dt;
  t->P = op->P;
  t->off = op->off;
  t->total = op->total;
  const size_t rsz = op->dt == QTT_F64 ? sizeof(double) : sizeof(float);
  if (cudaMalloc(&t->cores, rsz * op->total) != cudaSuccess) {
    cudaGetLastError();
    delete t;
    set_error("op_transpose: cudaMalloc");
    return QTT_ENOMEM;
  }
  for (int k = 1; k <= op->d; ++k) {
    const int P0 = op->P[k - 1], P1 = op->P[k];
    const int n = P0 * 4 * P1;
    if (op->dt == QTT_F64)
      op_transpose_kernel<double><<<(n + 255) / 256, 256, 0, s>>>(
          (const double*)op->cores + op->off[k - 1], (double*)t->cores + op->off[k - 1], P0, P1);
    else
      op_transpose_kernel<float><<<(n + 255) / 256, 256, 0, s>>>(
          (const float*)op->cores + op->off[k - 1], (float*)t->cores + op->off[k - 1], P0, P1);
  }
  qtt_status st = cuda_check(cudaGetLastError(), "op_transpose");
  if (st != QTT_OK) { op_free(t); return st; }
  *out = t;
  return QTT_OK;
}

}  // namespace qtt

extern "C" void qtt_debug_set_env_big(int on) { qtt::set_env_big(on); }
