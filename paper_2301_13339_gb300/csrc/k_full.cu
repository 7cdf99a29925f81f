// Full expansion (Alg. 3) and the QTT <-> array index maps (Sec. 4).
//
// Alg. 3 multiplies the cores left to right, the partial product growing to
// 2^{k-1} x r_{k-1} at step k.  Here the product is split at a cut a:
//   L  = X_1 ... X_a          (2^a x r_a, column-major, low bits fastest)
//   Rt = X_{a+1} ... X_d      (r_a x 2^{d-a})
//   y[lo + 2^a hi] = sum_alpha L[lo, alpha] Rt[alpha, hi]
// which is the same contraction regrouped; the last step is a dense
// 2^a x r_a x 2^{d-a} product streamed to HBM, stored through the QTT index
// -> array offset map (identity in 1D, bit de-interleave for 2D images).
// The offset of a QTT index q is linear in its bits, so
// offset(q) = off_lo[q mod 2^a] + off_hi[q / 2^a] with two small tables.
#include "qtt_internal.cuh"
#include <algorithm>
#include <atomic>

namespace qtt {

struct ModeMap {
  int d;
  int axis[32];   // 0 = x (fast array index), 1 = y
  int bit[32];
  int dx;         // log2 of the x extent (row length); 0 for 1D
};

static ModeMap make_mode_map(const TensorDesc& desc) {
  ModeMap mm{};
  mm.d = desc.d;
  if (desc.ndim == 1) {
    for (int k = 0; k < desc.d; ++k) { mm.axis[k] = 0; mm.bit[k] = k; }
    mm.dx = desc.d;
    return mm;
  }
  const int dy = desc.log2_shape[0], dx = desc.log2_shape[1];
  mm.dx = dx;
  int p = 0;
  if (desc.interleave) {
    for (int b = 0; b < std::max(dx, dy); ++b) {
      if (b < dx) { mm.axis[p] = 0; mm.bit[p] = b; ++p; }
      if (b < dy) { mm.axis[p] = 1; mm.bit[p] = b; ++p; }
    }
  } else {
    for (int b = 0; b < dx; ++b) { mm.axis[p] = 0; mm.bit[p] = b; ++p; }
    for (int b = 0; b < dy; ++b) { mm.axis[p] = 1; mm.bit[p] = b; ++p; }
  }
  return mm;
}

// offset table for modes [m0, m0 + nb): tab[u] = array offset of bits u
__global__ void offset_table_kernel(ModeMap mm, int m0, int nb, long long* tab) {
  const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= (1LL << nb)) return;
  long long x = 0, y = 0;
  for (int b = 0; b < nb; ++b) {
    const long long bitv = (u >> b) & 1;
    const int p = m0 + b;
    if (mm.axis[p] == 0) x |= bitv << mm.bit[p];
    else y |= bitv << mm.bit[p];
  }
  tab[u] = (y << mm.dx) + x;
}

// v[q] = img[off(q)]  (gather into QTT order)
template <typename T>
__global__ void morton_gather_kernel(const T* __restrict__ img, T* __restrict__ v,
                                     const long long* __restrict__ tlo,
                                     const long long* __restrict__ thi, int a, long long N) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  const long long lo = q & ((1LL << a) - 1), hi = q >> a;
  v[q] = img[tlo[lo] + thi[hi]];
}

template <typename T>
void launch_morton_gather(const T* img, T* v, int dx, int dy, int interleave, cudaStream_t s) {
  TensorDesc desc;
  desc.ndim = 2;
  desc.d = dx + dy;
  desc.log2_shape[0] = dy;
  desc.log2_shape[1] = dx;
  desc.interleave = interleave;
  ModeMap mm = make_mode_map(desc);
  const int d = desc.d;
  const int a = d / 2;
  long long* tlo = (long long*)scratch_alloc(sizeof(long long) << a, s);
  long long* thi = (long long*)scratch_alloc(sizeof(long long) << (d - a), s);
  offset_table_kernel<<<(int)(((1LL << a) + 255) / 256), 256, 0, s>>>(mm, 0, a, tlo);
  offset_table_kernel<<<(int)(((1LL << (d - a)) + 255) / 256), 256, 0, s>>>(mm, a, d - a, thi);
  const long long N = 1LL << d;
  QTT_PROF("morton_gather", s);
  morton_gather_kernel<T><<<(int)((N + 255) / 256), 256, 0, s>>>(img, v, tlo, thi, a, N);
  scratch_free(tlo, s);
  scratch_free(thi, s);
}
template void launch_morton_gather<double>(const double*, double*, int, int, int, cudaStream_t);
template void launch_morton_gather<float2>(const float2*, float2*, int, int, int, cudaStream_t);

// ---------------------------------------------------------------- partials
// Lout (2^k x r_k, ld 2^k) = Lin (2^{k-1} x r_{k-1}, ld 2^{k-1}) * core_k
// viewed as r_{k-1} x 2 r_k.  k = 1: Lin == nullptr and Lout = core_1.
template <typename T>
__global__ void left_partial_kernel(const T* __restrict__ Lin, const T* __restrict__ core,
                                    const int* __restrict__ ranks, int k, int rcapk,
                                    T* __restrict__ Lout) {
  const long long rows = 1LL << (k - 1);
  const int rp = ranks[k - 1], rk = ranks[k];
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * 2 * rcapk) return;
  const long long row = e % rows;
  const int col = (int)(e / rows);   // col = i + 2 beta
  if (col >= 2 * rk) return;
  T acc = szero<T>();
  if (Lin == nullptr) {
    acc = core[col];   // r_0 = 1
  } else {
    for (int al = 0; al < rp; ++al) mac(acc, Lin[row + rows * al], core[al + (size_t)rp * col]);
  }
  Lout[row + rows * col] = acc;
}

// Rout (r_{k-1} x 2^{d-k+1}, ld ldo) from core_k and Rin (r_k x 2^{d-k}, ld ldi);
// Rin == nullptr at k = d (Rout = core_d).
template <typename T>
__global__ void right_partial_kernel(const T* __restrict__ Rin, int ldi, const T* __restrict__ core,
                                     const int* __restrict__ ranks, int k, int d, int ldo,
                                     T* __restrict__ Rout) {
  const long long cols = 1LL << (d - k + 1);
  const int rp = ranks[k - 1], rk = ranks[k];
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)ldo * cols) return;
  const int al = (int)(e % ldo);
  const long long col = e / ldo;     // col = i + 2 rest
  if (al >= rp) return;
  const int i = (int)(col & 1);
  const long long rest = col >> 1;
  T acc = szero<T>();
  if (Rin == nullptr) {
    acc = core[al + (size_t)rp * i];
  } else {
    for (int be = 0; be < rk; ++be)
      mac(acc, core[al + (size_t)rp * (i + 2 * be)], Rin[be + (size_t)ldi * rest]);
  }
  Rout[al + (size_t)ldo * col] = acc;
}

// y[off_lo[lo] + off_hi[hi]] = sum_alpha L[lo + nlo alpha] Rt[alpha + ldr hi]
constexpr int FX_TL = 64, FX_TH = 64, FX_KC = 32;
template <typename T>
__global__ void __launch_bounds__(256)
expand_kernel(const T* __restrict__ L, long long nlo, const T* __restrict__ Rt, int ldr,
              long long nhi, const int* __restrict__ rptr, const long long* __restrict__ tlo,
              const long long* __restrict__ thi, const int* __restrict__ order64,
              T* __restrict__ y) {
  __shared__ T sL[FX_KC][FX_TL + 1];
  __shared__ T sR[FX_KC][FX_TH + 1];
  __shared__ T sO[FX_TH][FX_TL + 1];
  const int r = *rptr;
  const long long lo0 = (long long)blockIdx.x * FX_TL;
  const long long hi0 = (long long)blockIdx.y * FX_TH;
  const int tid = threadIdx.x;
  const int tl = (tid % 16) * 4, th = (tid / 16) * 4;
  T acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int z = 0; z < 4; ++z) acc[x][z] = szero<T>();
  for (int k0 = 0; k0 < r; k0 += FX_KC) {
    const int kc = min(FX_KC, r - k0);
    __syncthreads();
    for (int e = tid; e < FX_KC * FX_TL; e += 256) {
      const int l = e % FX_TL, kk = e / FX_TL;
      sL[kk][l] = (kk < kc && lo0 + l < nlo) ? L[(lo0 + l) + nlo * (k0 + kk)] : szero<T>();
    }
    for (int e = tid; e < FX_KC * FX_TH; e += 256) {
      const int kk = e % FX_KC, h = e / FX_KC;
      sR[kk][h] = (kk < kc && hi0 + h < nhi) ? Rt[(k0 + kk) + (size_t)ldr * (hi0 + h)] : szero<T>();
    }
    __syncthreads();
    for (int kk = 0; kk < kc; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) a[x] = sL[kk][tl + x];
#pragma unroll
      for (int z = 0; z < 4; ++z) b[z] = sR[kk][th + z];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int z = 0; z < 4; ++z) mac(acc[x][z], a[x], b[z]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int z = 0; z < 4; ++z) sO[th + z][tl + x] = acc[x][z];
  __syncthreads();
  // store: for each hi of the tile, the 64 lo in address order
  const long long base_lo = tlo[lo0];
  for (int e = tid; e < FX_TH * FX_TL; e += 256) {
    const int h = e / FX_TL, u = order64[e % FX_TL];
    if (lo0 + u < nlo && hi0 + h < nhi) y[base_lo + tlo[u] + thi[hi0 + h]] = sO[h][u];
  }
}

// order64[j] = the j-th of lo = 0..63 sorted by off_lo[lo]
__global__ void order64_kernel(const long long* tlo, int nlo_bits, int* order) {
  const int u = threadIdx.x;
  const int nu = 1 << min(nlo_bits, 6);
  if (u >= 64) return;
  if (u >= nu) { order[u] = u; return; }
  const long long ou = tlo[u];
  int rk = 0;
  for (int v = 0; v < nu; ++v) rk += (tlo[v] < ou) || (tlo[v] == ou && v < u);
  order[rk] = u;
}

// Cut of the Full split: the middle mode (even for an interleaved image, so
// that each half holds whole (x, y) bit pairs).
static int full_cut(const TensorDesc& desc) {
  int a = desc.d / 2;
  if (desc.ndim == 2 && desc.interleave) a &= ~1;
  return a < 1 ? 1 : a;
}

// Scratch of one expansion: left/right partial products (double-buffered)
// and the two offset tables.
template <typename T>
struct FullScratch {
  T* Lb0;
  T* Lb1;
  T* Rb0;
  T* Rb1;
  long long* tlo;
  long long* thi;
  int* order;
};

// The launch sequence of Full on caller-provided scratch: left partial
// X_1..X_a, right partial X_{a+1}..X_d, the two offset tables, the expansion.
template <typename T>
static qtt_status full_launch(const qtt_tensor* t, T* y, const FullScratch<T>& sc, cudaStream_t s) {
  const TensorDesc& desc = t->desc;
  const int d = desc.d;
  ModeMap mm = make_mode_map(desc);
  const int a = full_cut(desc);
  const long long nlo = 1LL << a, nhi = 1LL << (d - a);
  const T* cores = (const T*)t->cores;
  T* Lcur = nullptr;
  for (int k = 1; k <= a; ++k) {
    T* Lnext = (k & 1) ? sc.Lb0 : sc.Lb1;
    const long long tot = (1LL << (k - 1)) * 2 * t->rcap[k];
    QTT_PROF("full_partials", s);
    left_partial_kernel<T><<<(int)((tot + 255) / 256), 256, 0, s>>>(Lcur, cores + t->off[k - 1],
                                                                     t->ranks, k, t->rcap[k], Lnext);
    Lcur = Lnext;
  }
  T* Rcur = nullptr;
  int ldcur = 0;
  for (int k = d; k >= a + 1; --k) {
    T* Rnext = ((d - k) & 1) ? sc.Rb1 : sc.Rb0;
    const int ldo = t->rcap[k - 1];
    const long long tot = (long long)ldo << (d - k + 1);
    QTT_PROF("full_partials", s);
    right_partial_kernel<T><<<(int)((tot + 255) / 256), 256, 0, s>>>(
        Rcur, ldcur, cores + t->off[k - 1], t->ranks, k, d, ldo, Rnext);
    Rcur = Rnext;
    ldcur = ldo;
  }
  {
    QTT_PROF("full_partials", s);
    offset_table_kernel<<<(int)((nlo + 255) / 256), 256, 0, s>>>(mm, 0, a, sc.tlo);
    offset_table_kernel<<<(int)((nhi + 255) / 256), 256, 0, s>>>(mm, a, d - a, sc.thi);
    order64_kernel<<<1, 64, 0, s>>>(sc.tlo, a, sc.order);
  }
  dim3 grid((unsigned)((nlo + FX_TL - 1) / FX_TL), (unsigned)((nhi + FX_TH - 1) / FX_TH));
  {
    QTT_PROF("full_expand", s);
    // every output sample written once; 8 r_a flop each (complex) at the cut's capacity
    prof_add_work("full_expand", (Sc<T>::cplx ? 8.0 : 2.0) * t->rcap[a] * (double)nlo * nhi,
                  (double)nlo * nhi * sizeof(T));
    expand_kernel<T><<<grid, 256, 0, s>>>(Lcur, nlo, Rcur, ldcur, nhi, t->ranks + a, sc.tlo, sc.thi,
                                          sc.order, y);
  }
  return cuda_check(cudaGetLastError(), "to_full launch");
}

template <typename T>
static int full_rank_cap(const qtt_tensor* t) {
  int r = 1;
  for (int c : t->rcap) r = std::max(r, c);
  return r;
}

template <typename T>
qtt_status tt_full(const qtt_tensor* t, T* y, cudaStream_t s) {
  const int d = t->desc.d;
  const int a = full_cut(t->desc);
  const long long nlo = 1LL << a, nhi = 1LL << (d - a);
  const int rmaxcap = full_rank_cap<T>(t);
  FullScratch<T> sc;
  sc.Lb0 = (T*)scratch_alloc(sizeof(T) * nlo * rmaxcap, s);
  sc.Lb1 = (T*)scratch_alloc(sizeof(T) * nlo * rmaxcap, s);
  sc.Rb0 = (T*)scratch_alloc(sizeof(T) * nhi * rmaxcap, s);
  sc.Rb1 = (T*)scratch_alloc(sizeof(T) * nhi * rmaxcap, s);
  sc.tlo = (long long*)scratch_alloc(sizeof(long long) * nlo, s);
  sc.thi = (long long*)scratch_alloc(sizeof(long long) * nhi, s);
  sc.order = (int*)scratch_alloc(sizeof(int) * 64, s);
  auto release = [&]() {
    scratch_free(sc.Lb0, s); scratch_free(sc.Lb1, s); scratch_free(sc.Rb0, s);
    scratch_free(sc.Rb1, s); scratch_free(sc.tlo, s); scratch_free(sc.thi, s);
    scratch_free(sc.order, s);
  };
  if (!sc.Lb0 || !sc.Lb1 || !sc.Rb0 || !sc.Rb1 || !sc.tlo || !sc.thi || !sc.order) {
    release();
    set_error("to_full: scratch allocation failed");
    return QTT_ENOMEM;
  }
  const qtt_status st = full_launch<T>(t, y, sc, s);
  release();
  return st;
}
template qtt_status tt_full<double>(const qtt_tensor*, double*, cudaStream_t);
template qtt_status tt_full<float2>(const qtt_tensor*, float2*, cudaStream_t);

// --------------------------------------------------------------------------
// Allocation-free variant of Full for callers that must not allocate device
// memory after start-up: latency-critical loops where a cudaMalloc (which can
// synchronise the device and has unbounded latency) is not acceptable, and
// processes whose device memory is already reserved by another allocator,
// where a cudaMalloc could fail.  The scratch (left/right partial products,
// index tables) lives in the file-scope device array below; every GPU that
// loads the library holds it until the process exits.
constexpr size_t FULL_NOALLOC_SCRATCH_BYTES = 16u << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_full_noalloc_scratch[FULL_NOALLOC_SCRATCH_BYTES];

static constexpr int NOALLOC_MAX_DEVICES = 64;
static std::atomic<void*> g_noalloc_ptr[NOALLOC_MAX_DEVICES];

// Device address of the scratch array on the current device (looked up once
// per device with that device current; the host-side symbol is only a
// stand-in and must never be passed to a kernel).  The cache entries are
// atomic, so host threads making their first calls at the same time are
// safe (each may look the address up; all store the same value).
static qtt_status noalloc_scratch_ptr(void** out) {
  int dev = 0;
  qtt_status st = cuda_check(cudaGetDevice(&dev), "to_full_noalloc: cudaGetDevice");
  if (st != QTT_OK) return st;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    set_error("to_full_noalloc: device index %d not supported", dev);
    return QTT_EUNSUPPORTED;
  }
  void* p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    st = cuda_check(cudaGetSymbolAddress(&p, g_full_noalloc_scratch),
                    "to_full_noalloc: cudaGetSymbolAddress");
    if (st != QTT_OK) return st;
    g_noalloc_ptr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return QTT_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename T>
static qtt_status tt_full_noalloc_t(const qtt_tensor* t, T* y, cudaStream_t s) {
  const int d = t->desc.d;
  const int a = full_cut(t->desc);
  const long long nlo = 1LL << a, nhi = 1LL << (d - a);
  const int rmaxcap = full_rank_cap<T>(t);
  const size_t lb = align256(sizeof(T) * (size_t)nlo * rmaxcap);
  const size_t rb = align256(sizeof(T) * (size_t)nhi * rmaxcap);
  const size_t tl = align256(sizeof(long long) * (size_t)nlo);
  const size_t th = align256(sizeof(long long) * (size_t)nhi);
  const size_t need = 2 * lb + 2 * rb + tl + th + align256(sizeof(int) * 64);
  if (need > FULL_NOALLOC_SCRATCH_BYTES) {
    set_error("qtt_to_full_noalloc: needs %zu bytes of scratch, the static limit is %zu bytes "
              "(use qtt_to_full)", need, FULL_NOALLOC_SCRATCH_BYTES);
    return QTT_EINVAL;
  }
  void* base = nullptr;
  qtt_status st = noalloc_scratch_ptr(&base);
  if (st != QTT_OK) return st;
  char* p = (char*)base;
  FullScratch<T> sc;
  sc.Lb0 = (T*)p; p += lb;
  sc.Lb1 = (T*)p; p += lb;
  sc.Rb0 = (T*)p; p += rb;
  sc.Rb1 = (T*)p; p += rb;
  sc.tlo = (long long*)p; p += tl;
  sc.thi = (long long*)p; p += th;
  sc.order = (int*)p;
  // Every scratch element that is read is first written in this call, so
  // nothing has to be cleared between calls.
  return full_launch<T>(t, y, sc, s);
}

}  // namespace qtt

extern "C" qtt_status qtt_to_full_noalloc(const qtt_tensor* t, void* y, void* stream) {
  using namespace qtt;
  clear_error();
  if (!t || !y) {
    set_error("qtt_to_full_noalloc: NULL argument");
    return QTT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const qtt_status st = (t->desc.dt == QTT_F64) ? tt_full_noalloc_t<double>(t, (double*)y, s)
                                                : tt_full_noalloc_t<float2>(t, (float2*)y, s);
  tensor_stamp(t, s);   // records the handle's existing last-use event: no allocation
  return st;
}

