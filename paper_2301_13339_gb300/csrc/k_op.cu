// QTT Toeplitz operator of the sinc imaging kernel (plan-time).
//
// T[j, i] = c(j - i) with c(m) = h g(m h), g(x) = A sinc(pi B x) (Eq. GAF,
// Delta_x = 1/B), h = 2^-d, A = 1 / (h sum_m sinc(pi B m h)) when normalised
// (Eq. sinc_kern1 with the integral taken by the midpoint rule over the
// 2^{d+1}-1 grid offsets), A = 1 otherwise.
//
// QTT form (Toeplitz operators in QTT, cited in Sec. 1 as [KKT13]; derived
// here): with t = j - i + 2^d the generating vector chat[t] = c(t - 2^d)
// (chat[0] = 0) has d+1 QTT cores G_1..G_{d+1} (TT-SVD on the GPU, FP64,
// refined, at eps_op).  Subtracting i from j bit by bit with borrows b_k
// (b_1 = 0):  diff = j_k - i_k - b_k, t_k = diff mod 2, b_{k+1} = [diff < 0],
// and t_{d+1} = 1 - b_{d+1}.  Operator core k holds G_k[alpha, t_k, beta] at
// (b_k, alpha) -> (b_{k+1}, beta); the last core absorbs G_{d+1}.
#include "qtt_internal.cuh"
#include <algorithm>
#include <cmath>

namespace qtt {

__global__ void sinc_sum_kernel(long long n, double B, double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0.0;
  const long long tot = 2 * n - 1;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long m = e - (n - 1);
    if (m == 0) acc += 1.0;
    else {
      const double x = B * (double)m / (double)n;   // B m h
      acc += sinpi(x) / (M_PI * x);
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// *sum = the block partials added in a fixed order (lane l takes every 32nd
// partial from l, then a fixed shuffle tree): the same sum on every run,
// where an atomic accumulation would depend on the blocks' finishing order
__global__ void sinc_sum_finish(const double* __restrict__ part, int nparts, double* sum) {
  double t = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 32) t += part[i];
  for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
  if (threadIdx.x == 0) *sum = t;
}

// sum over m = -(n-1)..n-1 of sinc(pi B m / n) into *sum (device)
static qtt_status sinc_sum(long long n, double B, double* sum, cudaStream_t s) {
  const int blocks = (int)std::min<long long>((2 * n + 255) / 256, 4096);
  double* part = (double*)scratch_alloc(sizeof(double) * blocks, s);
  if (!part) return QTT_ENOMEM;
  sinc_sum_kernel<<<blocks, 256, 0, s>>>(n, B, part);
  sinc_sum_finish<<<1, 32, 0, s>>>(part, blocks, sum);
  scratch_free(part, s);
  return QTT_OK;
}

__global__ void chat_kernel(long long n, double B, int normalize, const double* sum,
                            double* chat) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * n) return;
  if (t == 0) { chat[0] = 0.0; return; }
  const long long m = t - n;
  double s;
  if (m == 0) s = 1.0;
  else {
    const double x = B * (double)m / (double)n;
    s = sinpi(x) / (M_PI * x);
  }
  // c(m) = h A sinc(pi B m h); normalised: h A = 1 / sum
  chat[t] = normalize ? s / (*sum) : s / (double)n;
}

// Sec. 2 padding of the kernel samples (the array g of Alg. 2): g[j] =
// c(j - (N-1)/2) for j < N (the kernel at the N grid points, centred), 0 for
// N <= j < n, with c(m) = h A sinc(pi B m h) normalised as in the operator
// plan (h = 1/n, h A = 1 / the sum over the 2n-1 offsets of the n-grid).
__device__ __forceinline__ void store_real(double& g, double v) { g = v; }
__device__ __forceinline__ void store_real(float2& g, double v) { g = make_float2((float)v, 0.f); }

template <typename T>
__global__ void sinc_padded_kernel(long long n, long long N, double B, int normalize,
                                   const double* __restrict__ sum, T* __restrict__ g) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double v = 0.0;
  if (j < N) {
    const long long m = j - (N - 1) / 2;
    double sv = 1.0;
    if (m != 0) {
      const double x = B * (double)m / (double)n;
      sv = sinpi(x) / (M_PI * x);
    }
    v = normalize ? sv / (*sum) : sv / (double)n;
  }
  store_real(g[j], v);
}

qtt_status sinc_padded(int log2_n, long long N, double B, int normalize, qtt_dtype dt, void* g,
                       cudaStream_t s) {
  const long long n = 1LL << log2_n;
  double* sum = (double*)scratch_alloc(sizeof(double), s);
  if (!sum) { set_error("qtt_sinc_padded: alloc"); return QTT_ENOMEM; }
  if (sinc_sum(n, B, sum, s) != QTT_OK) {
    scratch_free(sum, s);
    set_error("qtt_sinc_padded: alloc");
    return QTT_ENOMEM;
  }
  const int gb = (int)((n + 255) / 256);
  if (dt == QTT_F64) sinc_padded_kernel<double><<<gb, 256, 0, s>>>(n, N, B, normalize, sum, (double*)g);
  else sinc_padded_kernel<float2><<<gb, 256, 0, s>>>(n, N, B, normalize, sum, (float2*)g);
  scratch_free(sum, s);
  return cuda_check(cudaGetLastError(), "qtt_sinc_padded");
}

// One thread per operator core element; core k (1-based) of P_{k-1} x 2 x 2 x P_k,
// element (p, j, i, q) at p + P_{k-1} (j + 2 (i + 2 q)).
template <typename R>
__global__ void build_op_core_kernel(const double* __restrict__ Gk, int rho0, int rho1,
                                     const double* __restrict__ Glast, int rho_last_in,
                                     int k, int d, int Pin, int Pout, R* __restrict__ O) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int tot = Pin * 4 * Pout;
  if (e >= tot) return;
  const int p = e % Pin;
  const int j = (e / Pin) % 2;
  const int i = (e / (2 * Pin)) % 2;
  const int q = e / (4 * Pin);
  const int b = p / rho0, al = p % rho0;
  const int diff = j - i - b;
  const int t = diff & 1;
  const int bout = diff < 0 ? 1 : 0;
  double v = 0.0;
  if (k < d) {
    const int bq = q / rho1, be = q % rho1;
    if (bq == bout) v = Gk[al + rho0 * (t + 2 * be)];
  } else {
    // absorb G_{d+1}[beta, 1 - bout, 0] (rho_last_in = rho_d)
    for (int be = 0; be < rho1; ++be)
      v += Gk[al + rho0 * (t + 2 * be)] * Glast[be + rho_last_in * (1 - bout)];
  }
  O[e] = (R)v;
}

template <typename R>
__global__ void identity_core_kernel(int P, R* O) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= P * 4 * P) return;
  const int p = e % P, j = (e / P) % 2, i = (e / (2 * P)) % 2, q = e / (4 * P);
  O[e] = (R)((p == q && i == j) ? 1.0 : 0.0);
}

qtt_status op_sinc_create(int d, double B, int normalize, double eps_op, qtt_dtype dt,
                          cudaStream_t s, qtt_op** out) {
  if (d < 1 || d > 29) { set_error("op_sinc_create: d out of range"); return QTT_EINVAL; }
  const long long n = 1LL << d;
  double* sum = (double*)scratch_alloc(sizeof(double), s);
  double* chat = (double*)scratch_alloc(sizeof(double) * 2 * n, s);
  if (!sum || !chat) {
    scratch_free(sum, s);
    scratch_free(chat, s);
    set_error("op_sinc_create: alloc");
    return QTT_ENOMEM;
  }
  if (sinc_sum(n, B, sum, s) != QTT_OK) {
    scratch_free(sum, s);
    scratch_free(chat, s);
    set_error("op_sinc_create: alloc");
    return QTT_ENOMEM;
  }
  chat_kernel<<<(int)((2 * n + 255) / 256), 256, 0, s>>>(n, B, normalize, sum, chat);
  // TT-SVD of chat (d+1 modes), FP64 with refinement
  TensorDesc gd;
  gd.d = d + 1;
  gd.dt = QTT_F64;
  gd.ndim = 1;
  gd.log2_shape[0] = d + 1;
  qtt_tensor* G = nullptr;
  qtt_status st = tensor_alloc(gd, rank_caps(d + 1, 0, QTT_RANK_CAP), s, &G);
  if (st != QTT_OK) return st;
  qtt_trunc tr{eps_op, 0, 1, 0.0};
  st = tt_svd<double>(chat, d + 1, tr, G, s);
  if (st != QTT_OK) { qtt_free(G); return st; }
  std::vector<int> rho(d + 2);
  st = cuda_check(cudaMemcpyAsync(rho.data(), G->ranks, sizeof(int) * (d + 2),
                                  cudaMemcpyDeviceToHost, s), "op ranks");
  if (st != QTT_OK) { qtt_free(G); return st; }
  st = cuda_check(cudaStreamSynchronize(s), "op sync");
  if (st != QTT_OK) { qtt_free(G); return st; }
  qtt_op* op = new qtt_op();
  op->d = d;
  op->dt = dt;
  op->P.assign(d + 1, 1);
  for (int k = 1; k < d; ++k) op->P[k] = 2 * rho[k];
  op->off.resize(d);
  size_t tot = 0;
  for (int k = 0; k < d; ++k) {
    op->off[k] = tot;
    tot += (size_t)op->P[k] * 4 * op->P[k + 1];
  }
  op->total = tot;
  const size_t rsz = (dt == QTT_F64) ? sizeof(double) : sizeof(float);
  if (cudaMalloc(&op->cores, rsz * tot) != cudaSuccess) {
    cudaGetLastError();
    delete op;
    qtt_free(G);
    set_error("op_sinc_create: cudaMalloc");
    return QTT_ENOMEM;
  }
  const double* Gc = (const double*)G->cores;
  for (int k = 1; k <= d; ++k) {
    const int Pin = op->P[k - 1], Pout = op->P[k];
    const int cnt = Pin * 4 * Pout;
    const double* Gk = Gc + G->off[k - 1];
    const double* Glast = Gc + G->off[d];
    if (dt == QTT_F64)
      build_op_core_kernel<double><<<(cnt + 255) / 256, 256, 0, s>>>(
          Gk, rho[k - 1], rho[k], Glast, rho[d], k, d, Pin, Pout,
          (double*)op->cores + op->off[k - 1]);
    else
      build_op_core_kernel<float><<<(cnt + 255) / 256, 256, 0, s>>>(
          Gk, rho[k - 1], rho[k], Glast, rho[d], k, d, Pin, Pout,
          (float*)op->cores + op->off[k - 1]);
  }
  st = cuda_check(cudaStreamSynchronize(s), "op build");
  qtt_free(G);
  scratch_free(sum, s);
  scratch_free(chat, s);
  if (st != QTT_OK) { op_free(op); return st; }
  *out = op;
  return QTT_OK;
}

// Operator on all modes of an image for one axis: identity cores on the
// modes of the other axis carry the operator rank through unchanged.
qtt_status op_embed_axis(const qtt_op* op1d, const TensorDesc& desc, int axis, cudaStream_t s,
                         qtt_op** out) {
  const int dy = desc.log2_shape[0], dx = desc.log2_shape[1];
  std::vector<std::pair<int, int>> modes;
  if (desc.interleave) {
    for (int b = 0; b < std::max(dx, dy); ++b) {
      if (b < dx) modes.push_back({0, b});
      if (b < dy) modes.push_back({1, b});
    }
  } else {
    for (int b = 0; b < dx; ++b) modes.push_back({0, b});
    for (int b = 0; b < dy; ++b) modes.push_back({1, b});
  }
  const int d = (int)modes.size();
  qtt_op* op = new qtt_op();
  op->d = d;
  op->dt = op1d->dt;
  op->P.assign(d + 1, 1);
  int rank = 1;
  for (int p = 0; p < d; ++p) {
    if (modes[p].first == axis) rank = op1d->P[modes[p].second + 1];
    op->P[p + 1] = rank;
  }
  op->off.resize(d);
  size_t tot = 0;
  for (int k = 0; k < d; ++k) {
    op->off[k] = tot;
    tot += (size_t)op->P[k] * 4 * op->P[k + 1];
  }
  op->total = tot;
  const size_t rsz = (op->dt == QTT_F64) ? sizeof(double) : sizeof(float);
  if (cudaMalloc(&op->cores, rsz * tot) != cudaSuccess) {
    cudaGetLastError();
    delete op;
    set_error("op_embed_axis: cudaMalloc");
    return QTT_ENOMEM;
  }
  for (int p = 0; p < d; ++p) {
    char* dst = (char*)op->cores + rsz * op->off[p];
    if (modes[p].first == axis) {
      const int b = modes[p].second;
      const size_t cnt = (size_t)op1d->P[b] * 4 * op1d->P[b + 1];
      cudaMemcpyAsync(dst, (const char*)op1d->cores + rsz * op1d->off[b], rsz * cnt,
                      cudaMemcpyDeviceToDevice, s);
    } else {
      const int P = op->P[p];
      if (op->dt == QTT_F64)
        identity_core_kernel<double><<<(P * 4 * P + 255) / 256, 256, 0, s>>>(P, (double*)dst);
      else
        identity_core_kernel<float><<<(P * 4 * P + 255) / 256, 256, 0, s>>>(P, (float*)dst);
    }
  }
  qtt_status st = cuda_check(cudaGetLastError(), "op_embed_axis");
  if (st != QTT_OK) { op_free(op); return st; }
  *out = op;
  return QTT_OK;
}

void op_free(qtt_op* op) {
  if (!op) return;
  if (op->cores) cudaFree(op->cores);
  delete op;
}

// ---------------------------------------------------------------- matvec
// Y_k[(a + r_{k-1} p), j, (b + r_k q)] = sum_i O_k[p, j, i, q] X_k[a, i, b]
template <typename T, typename R>
__global__ void matvec_core_kernel(const R* __restrict__ O, int Pin, int Pout,
                                   const T* __restrict__ X, const int* __restrict__ xr, int k,
                                   int* __restrict__ yr, T* __restrict__ Y, long long capel) {
  const int r0 = xr[k - 1], r1 = xr[k];
  const int R0 = Pin * r0, R1 = Pout * r1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    yr[k] = R1;
    if (k == 1) yr[0] = R0;
  }
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)R0 * 2 * R1 || e >= capel) return;
  const int c0 = (int)(e % R0);
  const int j = (int)((e / R0) % 2);
  const int c1 = (int)(e / (2LL * R0));
  const int a = c0 % r0, p = c0 / r0;
  const int b = c1 % r1, q = c1 / r1;
  T acc = szero<T>();
  for (int i = 0; i < 2; ++i)
    rmac(acc, O[p + Pin * (j + 2 * (i + 2 * q))], X[a + (size_t)r0 * (i + 2 * b)]);
  Y[e] = acc;
}

qtt_status matvec(const qtt_op* op, const qtt_tensor* x, cudaStream_t s, qtt_tensor** out) {
  const int d = x->desc.d;
  if (op->d != d) { set_error("matvec: operator has %d modes, tensor %d", op->d, d); return QTT_EINVAL; }
  if (op->dt != x->desc.dt) { set_error("matvec: operator/tensor dtype mismatch"); return QTT_EINVAL; }
  if (op->cplx && x->desc.dt != QTT_C64) { set_error("matvec: complex operator on a real tensor"); return QTT_EINVAL; }
  std::vector<int> cap(d + 1);
  for (int k = 0; k <= d; ++k) {
    cap[k] = op->P[k] * x->rcap[k];
    if (cap[k] > QTT_PRODUCT_CAP) {
      set_error("matvec: product rank capacity %d above %d", cap[k], QTT_PRODUCT_CAP);
      return QTT_EINVAL;
    }
  }
  qtt_tensor* y = nullptr;
  qtt_status st = tensor_alloc(x->desc, cap, s, &y);
  if (st != QTT_OK) return st;
  for (int k = 1; k <= d; ++k) {
    const long long capel = (long long)cap[k - 1] * 2 * cap[k];
    const int blocks = (int)((capel + 255) / 256);
    if (x->desc.dt == QTT_F64)
      matvec_core_kernel<double, double><<<blocks, 256, 0, s>>>(
          (const double*)op->cores + op->off[k - 1], op->P[k - 1], op->P[k],
          (const double*)x->cores + x->off[k - 1], x->ranks, k, y->ranks,
          (double*)y->cores + y->off[k - 1], capel);
    else if (op->cplx)
      matvec_core_kernel<float2, float2><<<blocks, 256, 0, s>>>(
          (const float2*)op->cores + op->off[k - 1], op->P[k - 1], op->P[k],
          (const float2*)x->cores + x->off[k - 1], x->ranks, k, y->ranks,
          (float2*)y->cores + y->off[k - 1], capel);
    else
      matvec_core_kernel<float2, float><<<blocks, 256, 0, s>>>(
          (const float*)op->cores + op->off[k - 1], op->P[k - 1], op->P[k],
          (const float2*)x->cores + x->off[k - 1], x->ranks, k, y->ranks,
          (float2*)y->cores + y->off[k - 1], capel);
  }
  st = cuda_check(cudaGetLastError(), "matvec");
  if (st != QTT_OK) { qtt_free(y); return st; }
  *out = y;
  return QTT_OK;
}

}  // namespace qtt
