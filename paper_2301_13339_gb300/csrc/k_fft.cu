// QTT-FFT / QTT-iFFT (Sec. 4, the QTT-FFT of [DKS12]; truncated as in Sec. 5)
// and the entrywise (Hadamard) product of Alg. 2 Step 3.
//
// The transform is the radix-2 decimation-in-frequency FFT with one QTT
// operator per bit.  For an axis whose bit b+1 sits on mode modes[b]
// (increasing), the stage on bit p maps the pair (x_n, x_{n + 2^(p-1)}) of
// each size-2^p sub-transform to (x_n + x_{n+2^(p-1)},
// (x_n - x_{n+2^(p-1)}) w^n), w = exp(-+2 pi i / 2^p), n = the lower p-1
// bits.  As a TT operator (cores O[l, out, in, r], column-major, bonds in
// {1, 2}):
//   mode modes[p-1]        butterfly [[1, 1], [1, -1]]; for p > 1 the new bit
//                          leaves to the left as the branch c (bond 2);
//   mode modes[b], b < p-1 twiddle w^(i 2^b) on branch c = 1, 1 on c = 0;
//   other modes between    the branch passes through (bond 2, identity);
//   every other mode       identity (bond 1).
// The inverse stage uses exp(+...) and halves the butterfly, so that the d
// stages carry the 1/N^D of the inverse DFT.  Each stage is applied by the
// operator x vector contraction (k_op.cu, complex operator cores) and
// followed by TT-rounding (k_round.cu) with the caller's truncation (cap
// R^_max, tolerance or SV drop-off); the input is rounded first.  After all
// stages bit b of an axis sits on the mode of its bit K-1-b; reversing the
// chain of cores (mode k <- mode d+1-k, bonds swapped) restores the natural
// order of every axis and mirrors the axes' positions: a 2D plain chain
// comes out with its blocks swapped, an interleaved square chain with the
// other axis first -- the layout of the transposed image.
#include "qtt_internal.cuh"
#include <algorithm>
#include <cmath>

namespace qtt {

constexpr int FFT_MAXD = 32;          // modes an axis descriptor can hold
constexpr int FFT_CORE_STRIDE = 16;   // elements reserved per stage core (2 x 2 x 2 x 2)

struct FftAxis {
  int d;                 // modes of the chain
  int K;                 // bits of this axis
  int inverse;           // 1: exp(+...) twiddles and a halved butterfly
  int modes[FFT_MAXD];   // 1-based mode of bit b+1, increasing
};

// Bond of cut c (0..d; cut c lies between modes c and c+1) of the stage on
// bit p: 2 from the axis' first bit up to, not including, bit p.
__host__ __device__ inline int fft_stage_bond(const int* modes, int p, int c) {
  return (c >= modes[0] && c < modes[p - 1]) ? 2 : 1;
}

// All K stage operators of one axis: stage p (blockIdx.y = p - 1) at
// O + (p - 1) d 16, its core on mode m at + (m - 1) 16, element
// [l, j, i, q] at l + Pin (j + 2 (i + 2 q)).
__global__ void fft_stage_ops_kernel(FftAxis ax, float2* __restrict__ O) {
  const int p = blockIdx.y + 1;
  const int d = ax.d;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d * FFT_CORE_STRIDE) return;
  const int m = t / FFT_CORE_STRIDE + 1;
  const int e = t % FFT_CORE_STRIDE;
  float2* Ok = O + ((size_t)blockIdx.y * d + (m - 1)) * FFT_CORE_STRIDE;
  const int Pin = fft_stage_bond(ax.modes, p, m - 1), Pout = fft_stage_bond(ax.modes, p, m);
  if (e >= Pin * 4 * Pout) {
    Ok[e] = make_float2(0.f, 0.f);
    return;
  }
  const int l = e % Pin, j = (e / Pin) % 2, i = (e / (2 * Pin)) % 2, q = e / (4 * Pin);
  const int lo = ax.modes[0], hi = ax.modes[p - 1];
  int bit = 0;                              // bit of this axis held by mode m, below p (0: none)
  for (int b = 0; b < p - 1; ++b)
    if (ax.modes[b] == m) bit = b + 1;
  double re = 0.0, im = 0.0;
  if (m == hi) {
    if (p == 1 || l == j) re = (ax.inverse ? 0.5 : 1.0) * ((j == 1 && i == 1) ? -1.0 : 1.0);
  } else if (bit > 0) {
    if (i == j && (Pin == 1 || l == q)) {
      if (q == 0 || i == 0) {
        re = 1.0;
      } else {
        // w^(2^(bit-1)) = exp(-+ i pi 2^(bit - p))
        const double a = (ax.inverse ? 1.0 : -1.0) * ldexp(1.0, bit - p);
        sincospi(a, &im, &re);
      }
    }
  } else if (m > lo && m < hi) {
    if (i == j && l == q) re = 1.0;
  } else {
    if (i == j) re = 1.0;
  }
  Ok[e] = make_float2((float)re, (float)im);
}

// Core k (1-based) of X becomes core d+1-k of Y with its bonds swapped:
// Y[b, i, a] = X[a, i, b].  Thread 0 writes the ranks of Y's cuts d-k and
// (for k = 1) d.
template <typename T>
__global__ void reverse_core_kernel(const T* __restrict__ X, const int* __restrict__ xr, int k,
                                    int d, int* __restrict__ yr, T* __restrict__ Y,
                                    long long capel) {
  const int r0 = xr[k - 1], r1 = xr[k];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    yr[d - k] = r1;
    if (k == 1) yr[d] = r0;
  }
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)r1 * 2 * r0 || e >= capel) return;
  const int b = (int)(e % r1);
  const int i = (int)((e / r1) % 2);
  const int a = (int)(e / (2LL * r1));
  Y[e] = X[a + (size_t)r0 * (i + 2 * b)];
}

__device__ __forceinline__ void mul_into(double& z, double a, double b) { z = a * b; }
__device__ __forceinline__ void mul_into(float2& z, float2 a, float2 b) {
  z.x = fmaf(a.x, b.x, -a.y * b.y);
  z.y = fmaf(a.x, b.y, a.y * b.x);
}

// Z_k[(a + ra a'), i, (b + rb b')] = A_k[a, i, b] B_k[a', i, b']
template <typename T>
__global__ void hadamard_core_kernel(const T* __restrict__ A, const int* __restrict__ ar,
                                     const T* __restrict__ B, const int* __restrict__ br, int k,
                                     int* __restrict__ zr, T* __restrict__ Z, long long capel) {
  const int a0 = ar[k - 1], a1 = ar[k], b0 = br[k - 1], b1 = br[k];
  const int R0 = a0 * b0, R1 = a1 * b1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    zr[k] = R1;
    if (k == 1) zr[0] = R0;
  }
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)R0 * 2 * R1 || e >= capel) return;
  const int c0 = (int)(e % R0);
  const int i = (int)((e / R0) % 2);
  const int c1 = (int)(e / (2LL * R0));
  const int a = c0 % a0, a2 = c0 / a0;
  const int b = c1 % a1, b2 = c1 / a1;
  T z;
  mul_into(z, A[a + (size_t)a0 * (i + 2 * b)], B[a2 + (size_t)b0 * (i + 2 * b2)]);
  Z[e] = z;
}

// dst |= src (device status words of two handles)
__global__ void status_or_kernel(int* __restrict__ dst, const int* __restrict__ src) {
  if (threadIdx.x == 0) atomicOr(dst, *src);
}

static void status_or(qtt_tensor* dst, const qtt_tensor* src, cudaStream_t s) {
  status_or_kernel<<<1, 32, 0, s>>>(dst->status, src->status);
}

qtt_status hadamard(const qtt_tensor* x, const qtt_tensor* y, cudaStream_t s, qtt_tensor** out) {
  const int d = x->desc.d;
  std::vector<int> cap(d + 1);
  for (int c = 0; c <= d; ++c) {
    cap[c] = x->rcap[c] * y->rcap[c];
    if (cap[c] > QTT_PRODUCT_CAP) {
      set_error("hadamard: product rank capacity %d above %d", cap[c], QTT_PRODUCT_CAP);
      return QTT_EINVAL;
    }
  }
  qtt_tensor* z = nullptr;
  qtt_status st = tensor_alloc(x->desc, cap, s, &z);
  if (st != QTT_OK) return st;
  for (int k = 1; k <= d; ++k) {
    const long long capel = (long long)cap[k - 1] * 2 * cap[k];
    const int blocks = (int)((capel + 255) / 256);
    if (x->desc.dt == QTT_F64)
      hadamard_core_kernel<double><<<blocks, 256, 0, s>>>(
          (const double*)x->cores + x->off[k - 1], x->ranks, (const double*)y->cores + y->off[k - 1],
          y->ranks, k, z->ranks, (double*)z->cores + z->off[k - 1], capel);
    else
      hadamard_core_kernel<float2><<<blocks, 256, 0, s>>>(
          (const float2*)x->cores + x->off[k - 1], x->ranks, (const float2*)y->cores + y->off[k - 1],
          y->ranks, k, z->ranks, (float2*)z->cores + z->off[k - 1], capel);
  }
  status_or(z, x, s);
  status_or(z, y, s);
  st = cuda_check(cudaGetLastError(), "hadamard");
  if (st != QTT_OK) { tensor_free_async(z, s); return st; }
  *out = z;
  return QTT_OK;
}

// The axes of a layout, in the order the transform takes them (by the mode
// of each axis' least significant bit), and the layout of the result.
static qtt_status fft_axes(const TensorDesc& in, std::vector<std::vector<int>>& axes,
                           TensorDesc& outd) {
  const int d = in.d;
  axes.clear();
  outd = in;
  if (in.ndim == 1) {
    std::vector<int> a(d);
    for (int b = 0; b < d; ++b) a[b] = b + 1;
    axes.push_back(a);
    return QTT_OK;
  }
  const int dy = in.log2_shape[0], dx = in.log2_shape[1];
  std::vector<int> ax, ay;
  if (!in.interleave) {
    for (int b = 0; b < dx; ++b) ax.push_back(b + 1);
    for (int b = 0; b < dy; ++b) ay.push_back(dx + b + 1);
  } else {
    if (dx != dy) {
      set_error("qtt_fft: an interleaved 2D layout needs equal axes (got 2^%d x 2^%d)", dy, dx);
      return QTT_EUNSUPPORTED;
    }
    for (int b = 0; b < dx; ++b) {
      ax.push_back(2 * b + 1);
      ay.push_back(2 * b + 2);
    }
  }
  axes.push_back(ax);
  axes.push_back(ay);
  outd.log2_shape[0] = dx;
  outd.log2_shape[1] = dy;
  return QTT_OK;
}

qtt_status fft_transform(const qtt_tensor* x, int inverse, const qtt_trunc& tr, const qtt_op* id,
                         int sketch, unsigned long long seed, cudaStream_t s, qtt_tensor** out) {
  const int d = x->desc.d;
  if (x->desc.dt != QTT_C64) {
    set_error("qtt_fft: a spectrum needs a complex handle (QTT_C64)");
    return QTT_EUNSUPPORTED;
  }
  if (d > FFT_MAXD) { set_error("qtt_fft: %d modes above %d", d, FFT_MAXD); return QTT_EINVAL; }
  std::vector<std::vector<int>> axes;
  TensorDesc od;
  qtt_status st = fft_axes(x->desc, axes, od);
  if (st != QTT_OK) return st;

  qtt_tensor* y = nullptr;
  {
    QTT_PROF("fft_round", s);
    st = round_product(id, x, tr, sketch, seed, s, &y);
  }
  if (st != QTT_OK) return st;
  status_or(y, x, s);
  unsigned long long stage_seed = seed;
  for (const std::vector<int>& modes : axes) {
    const int K = (int)modes.size();
    FftAxis A;
    A.d = d;
    A.K = K;
    A.inverse = inverse ? 1 : 0;
    for (int b = 0; b < FFT_MAXD; ++b) A.modes[b] = b < K ? modes[b] : 0;
    float2* O = (float2*)scratch_alloc(sizeof(float2) * (size_t)K * d * FFT_CORE_STRIDE, s);
    if (!O) {
      tensor_free_async(y, s);
      set_error("qtt_fft: out of device memory for the stage operators");
      return QTT_ENOMEM;
    }
    fft_stage_ops_kernel<<<dim3((d * FFT_CORE_STRIDE + 127) / 128, K), 128, 0, s>>>(A, O);
    for (int p = K; p >= 1 && st == QTT_OK; --p) {
      qtt_op op;
      op.d = d;
      op.dt = QTT_C64;
      op.cplx = 1;
      op.P.resize(d + 1);
      for (int c = 0; c <= d; ++c) op.P[c] = fft_stage_bond(modes.data(), p, c);
      op.off.resize(d);
      for (int k = 0; k < d; ++k) op.off[k] = (size_t)k * FFT_CORE_STRIDE;
      op.total = (size_t)d * FFT_CORE_STRIDE;
      op.cores = O + (size_t)(p - 1) * d * FFT_CORE_STRIDE;
      qtt_tensor* z = nullptr;
      {
        QTT_PROF("fft_stage", s);
        st = matvec(&op, y, s, &z);
      }
      op.cores = nullptr;
      if (st != QTT_OK) break;
      status_or(z, y, s);
      tensor_free_async(y, s);
      y = nullptr;
      {
        QTT_PROF("fft_round", s);
        st = round_product(id, z, tr, sketch, ++stage_seed, s, &y);
      }
      if (st == QTT_OK) status_or(y, z, s);
      tensor_free_async(z, s);
    }
    scratch_free(O, s);
    if (st != QTT_OK) {
      if (y) tensor_free_async(y, s);
      return st;
    }
  }

  std::vector<int> rc(d + 1);
  for (int c = 0; c <= d; ++c) rc[c] = y->rcap[d - c];
  qtt_tensor* r = nullptr;
  st = tensor_alloc(od, rc, s, &r);
  if (st != QTT_OK) { tensor_free_async(y, s); return st; }
  for (int k = 1; k <= d; ++k) {
    const long long capel = (long long)y->rcap[k - 1] * 2 * y->rcap[k];
    const int blocks = (int)((capel + 255) / 256);
    reverse_core_kernel<float2><<<blocks, 256, 0, s>>>(
        (const float2*)y->cores + y->off[k - 1], y->ranks, k, d, r->ranks,
        (float2*)r->cores + r->off[d - k], capel);
  }
  status_or(r, y, s);
  tensor_free_async(y, s);
  st = cuda_check(cudaGetLastError(), "qtt_fft");
  if (st != QTT_OK) { tensor_free_async(r, s); return st; }
  *out = r;
  return QTT_OK;
}

}  // namespace qtt
