// C ABI of libqtt: argument checks, handle management, operator plan cache.
// The numerical work is in k_svd.cu (TT-SVD), k_op.cu (operator plan and
// matvec), k_round.cu (rounding of operator x vector), k_full.cu (Full) and
// k_fft.cu (QTT-FFT stages, Hadamard product).
#include "qtt_internal.cuh"
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <algorithm>

namespace qtt {

static thread_local char g_err[512] = "";

void clear_error() { g_err[0] = 0; }

int device_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return 1;
  }
  return n;
}

bool first_on_device(std::atomic<unsigned long long>* flags) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return true;
  const unsigned long long bit = 1ull << dev;
  return (flags->fetch_or(bit) & bit) == 0;
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

qtt_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return QTT_OK;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? QTT_ENOMEM : QTT_ECUDA;
}

size_t elem_size(qtt_dtype dt) { return dt == QTT_F64 ? sizeof(double) : sizeof(float2); }

static std::once_flag g_pool_once;
static void configure_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    // keep freed blocks in the pool between calls (process-local setting)
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
}

void* scratch_alloc(size_t bytes, cudaStream_t s) {
  std::call_once(g_pool_once, configure_pool);
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void scratch_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

std::vector<int> rank_caps(int d, int rmax, int cap) {
  std::vector<int> r(d + 1, 1);
  const int lim = (rmax > 0) ? std::min(rmax, cap) : cap;
  for (int k = 1; k < d; ++k) {
    long long a = 1LL << std::min(k, 40), b = 1LL << std::min(d - k, 40);
    r[k] = (int)std::min<long long>({a, b, (long long)lim});
  }
  return r;
}

struct RankList {
  int v[34];
};
__global__ void set_ranks_kernel(int* dst, RankList rl, int n) {
  const int i = threadIdx.x;
  if (i < n) dst[i] = rl.v[i];
}

void set_ranks_from_host(int* dev_ranks, const std::vector<int>& r, cudaStream_t s) {
  RankList rl{};
  const int n = (int)std::min<size_t>(r.size(), 34);
  for (int i = 0; i < n; ++i) rl.v[i] = r[i];
  set_ranks_kernel<<<1, 64, 0, s>>>(dev_ranks, rl, n);
}

qtt_status tensor_alloc(const TensorDesc& desc, const std::vector<int>& rcap, cudaStream_t s,
                        qtt_tensor** out) {
  const int d = desc.d;
  qtt_tensor* t = new qtt_tensor();
  t->desc = desc;
  t->rcap = rcap;
  t->off.resize(d);
  size_t tot = 0;
  for (int k = 0; k < d; ++k) {
    t->off[k] = tot;
    tot += (size_t)rcap[k] * 2 * rcap[k + 1];
  }
  t->total = tot;
  const size_t esz = elem_size(desc.dt);
  size_t core_bytes = (tot * esz + 255) & ~(size_t)255;
  size_t meta = 256 + 64 + 320;  // ranks (<= 33 ints -> 256 B), status, norm2, margins
  char* base = (char*)scratch_alloc(core_bytes + meta, s);
  if (!base) {
    delete t;
    set_error("tensor_alloc: out of device memory (%zu bytes)", core_bytes + meta);
    return QTT_ENOMEM;
  }
  t->cores = base;
  t->ranks = (int*)(base + core_bytes);
  t->status = (int*)(base + core_bytes + 256);
  t->norm2 = (double*)(base + core_bytes + 256 + 8);
  t->margin = (double*)(base + core_bytes + 320);
  cudaMemsetAsync(base + core_bytes, 0, 320, s);
  cudaMemsetAsync(base + core_bytes + 320, 0xff, meta - 320, s);   // NaN: no decision yet
  if (cudaEventCreateWithFlags(&t->used, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    t->used = nullptr;
  }
  tensor_stamp(t, s);
  *out = t;
  return QTT_OK;
}

void tensor_stamp(const qtt_tensor* t, cudaStream_t s) {
  if (!t || !t->used) return;
  // no stamp while s is being captured into a CUDA graph: the event would
  // become a node of the graph and must not be destroyed with the handle;
  // inside a graph the release is ordered by the graph itself
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (cs == cudaStreamCaptureStatusNone) cudaEventRecord(t->used, s);
}

void tensor_free_async(qtt_tensor* t, cudaStream_t s) {
  if (!t) return;
  scratch_free(t->cores, s);
  if (t->used) cudaEventDestroy(t->used);
  delete t;
}

// the QTT-FFT route's calls: small eigen-solves check and repair themselves
struct RepairScope {
  RepairScope() { set_heev_repair(1); }
  ~RepairScope() { set_heev_repair(0); }
};

// The handles a C-ABI call uses, stamped on its stream when the call returns
// (after everything it enqueued), so that qtt_free can order the release
// after the last use without synchronising the device.
struct Touch {
  cudaStream_t s;
  const qtt_tensor* a;
  const qtt_tensor* b;
  qtt_tensor** out;
  ~Touch() {
    tensor_stamp(a, s);
    tensor_stamp(b, s);
    if (out) tensor_stamp(*out, s);
  }
};

// per-device stream on which qtt_free releases storage after the handle's
// last-use event
static cudaStream_t free_stream() {
  static std::mutex mu;
  static cudaStream_t streams[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    streams[dev] = nullptr;
  }
  return streams[dev];
}

// ---------------------------------------------------------------- op cache
typedef std::tuple<int, double, int, double, int> OpKey;  // d, B, normalize, eps_op, dt
typedef std::tuple<int, double, int, double, int, int, int, int, int> EmbKey;  // + dy, dx, inter, axis
static std::mutex g_cache_mu;
static std::map<OpKey, qtt_op*> g_op_cache;
static std::map<EmbKey, qtt_op*> g_emb_cache;
static std::map<std::pair<int, int>, qtt_op*> g_id_cache;
static std::map<const qtt_op*, qtt_op*> g_tr_cache;   // forward operator -> its transpose

static qtt_status cached_transpose(const qtt_op* op, cudaStream_t s, qtt_op** out) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto it = g_tr_cache.find(op);
  if (it != g_tr_cache.end()) { *out = it->second; return QTT_OK; }
  qtt_op* t = nullptr;
  qtt_status st = op_transpose(op, s, &t);
  if (st != QTT_OK) return st;
  g_tr_cache[op] = t;
  *out = t;
  return QTT_OK;
}

static qtt_status cached_op(int d, double B, int normalize, double eps_op, qtt_dtype dt,
                            cudaStream_t s, qtt_op** out) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  OpKey key(d, B, normalize, eps_op, (int)dt);
  auto it = g_op_cache.find(key);
  if (it != g_op_cache.end()) { *out = it->second; return QTT_OK; }
  qtt_op* op = nullptr;
  qtt_status st = op_sinc_create(d, B, normalize, eps_op, dt, s, &op);
  if (st != QTT_OK) return st;
  g_op_cache[key] = op;
  *out = op;
  return QTT_OK;
}

qtt_status cached_op_plan(int d, double B, int normalize, double eps_op, qtt_dtype dt,
                          cudaStream_t s, qtt_op** out) {
  return cached_op(d, B, normalize ? 1 : 0, eps_op, dt, s, out);
}

static qtt_status cached_embed(const TensorDesc& desc, int axis, double B, int normalize,
                               double eps_op, cudaStream_t s, qtt_op** out) {
  const int dax = desc.log2_shape[axis == 0 ? 1 : 0];
  qtt_op* op1 = nullptr;
  qtt_status st = cached_op(dax, B, normalize, eps_op, desc.dt, s, &op1);
  if (st != QTT_OK) return st;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  EmbKey key(dax, B, normalize, eps_op, (int)desc.dt, desc.log2_shape[0], desc.log2_shape[1],
             desc.interleave, axis);
  auto it = g_emb_cache.find(key);
  if (it != g_emb_cache.end()) { *out = it->second; return QTT_OK; }
  qtt_op* op = nullptr;
  st = op_embed_axis(op1, desc, axis, s, &op);
  if (st != QTT_OK) return st;
  g_emb_cache[key] = op;
  *out = op;
  return QTT_OK;
}

template <typename R>
__global__ void identity_op_kernel(R* O, int d) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 4 * d) return;
  const int j = e % 2, i = (e / 2) % 2;
  O[e] = (R)(i == j ? 1.0 : 0.0);
}

static qtt_status cached_identity(int d, qtt_dtype dt, cudaStream_t s, qtt_op** out) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto key = std::make_pair(d, (int)dt);
  auto it = g_id_cache.find(key);
  if (it != g_id_cache.end()) { *out = it->second; return QTT_OK; }
  qtt_op* op = new qtt_op();
  op->d = d;
  op->dt = dt;
  op->P.assign(d + 1, 1);
  op->off.resize(d);
  for (int k = 0; k < d; ++k) op->off[k] = 4 * (size_t)k;
  op->total = 4 * (size_t)d;
  const size_t rsz = dt == QTT_F64 ? sizeof(double) : sizeof(float);
  if (cudaMalloc(&op->cores, rsz * op->total) != cudaSuccess) {
    delete op;
    set_error("identity operator: cudaMalloc");
    return QTT_ENOMEM;
  }
  if (dt == QTT_F64) identity_op_kernel<double><<<1, 128, 0, s>>>((double*)op->cores, d);
  else identity_op_kernel<float><<<1, 128, 0, s>>>((float*)op->cores, d);
  g_id_cache[key] = op;
  *out = op;
  return QTT_OK;
}

// Truncation parameters of a call on data of type dt with d modes (d <= 0:
// not known here, the forced ranks are checked later); tt_svd: the call is
// a TT-SVD (the TF32-refined mode exists there, for complex64).
static qtt_status check_trunc(const qtt_trunc* tr, qtt_dtype dt, int d, bool tt_svd = false) {
  if (!tr) { set_error("truncation parameters are NULL"); return QTT_EINVAL; }
  if (!(tr->eps >= 0.0) || tr->eps >= 1.0) { set_error("eps must be in [0, 1)"); return QTT_EINVAL; }
  if (tr->delta >= 1.0 || tr->delta != tr->delta) { set_error("delta must be < 1 (<= 0: off)"); return QTT_EINVAL; }
  if (tr->prec < QTT_PREC_AUTO || tr->prec > QTT_PREC_TF32_REFINED) {
    set_error("prec %d is not a qtt_prec value", tr->prec);
    return QTT_EINVAL;
  }
  if (tr->prec == QTT_PREC_TF32_REFINED && !(tt_svd && dt == QTT_C64)) {
    set_error("the TF32-refined mode is built for the complex64 TT-SVD (qtt_decompose) only");
    return QTT_EUNSUPPORTED;
  }
  if (tr->prec == QTT_PREC_BF16_REFINED) {
    set_error("the BF16-refined tensor-core mode is not built");
    return QTT_EUNSUPPORTED;
  }
  if ((tr->prec == QTT_PREC_FP64 && dt != QTT_F64) || (tr->prec == QTT_PREC_FP32 && dt != QTT_C64)) {
    set_error("prec %d does not match the element type %d (FP64 arithmetic for QTT_F64, FP32 for "
              "QTT_C64)", tr->prec, (int)dt);
    return QTT_EINVAL;
  }
  if (tr->fixed_ranks && d > 0) {
    const int* r = tr->fixed_ranks;
    if (r[0] != 1 || r[d] != 1) { set_error("fixed_ranks: r_0 and r_d must be 1"); return QTT_EINVAL; }
    for (int k = 1; k < d; ++k) {
      const long long lim = std::min<long long>({1LL << std::min(k, 40), 1LL << std::min(d - k, 40),
                                                 (long long)QTT_RANK_CAP});
      if (r[k] < 1 || r[k] > lim) {
        set_error("fixed_ranks: r_%d = %d outside [1, %lld]", k, r[k], lim);
        return QTT_EINVAL;
      }
    }
  }
  return QTT_OK;
}

static bool valid_dtype(qtt_dtype dt) { return dt == QTT_F64 || dt == QTT_C64; }

// QTT_EUNSUPPORTED for the storage types this build does not compute with,
// QTT_EINVAL for values outside qtt_dtype
static qtt_status dtype_status(qtt_dtype dt, const char* who) {
  if (valid_dtype(dt)) return QTT_OK;
  if (dt == QTT_F32 || dt == QTT_C128) {
    set_error("%s: element type %d is not built (QTT_F64 and QTT_C64 are)", who, (int)dt);
    return QTT_EUNSUPPORTED;
  }
  set_error("%s: unsupported dtype %d", who, (int)dt);
  return QTT_EINVAL;
}

}  // namespace qtt

using namespace qtt;

extern "C" {

const char* qtt_last_error(void) { return g_err; }
const char* qtt_version(void) { return "qtt-gb300 0.1 (sm_103a)"; }

qtt_status qtt_decompose(const void* x, qtt_dtype dt, int ndim, const int* log2_shape,
                         int interleave, const qtt_trunc* tr, void* stream, qtt_tensor** out) {
  g_err[0] = 0;
  if (!x || !log2_shape || !out) { set_error("qtt_decompose: NULL argument"); return QTT_EINVAL; }
  Touch tg{(cudaStream_t)stream, nullptr, nullptr, out};
  qtt_status st = dtype_status(dt, "qtt_decompose");
  if (st != QTT_OK) return st;
  if (ndim != 1 && ndim != 2) { set_error("qtt_decompose: ndim must be 1 or 2"); return QTT_EINVAL; }
  st = check_trunc(tr, dt, 0, true);
  if (st != QTT_OK) return st;
  TensorDesc desc;
  desc.dt = dt;
  desc.ndim = ndim;
  desc.interleave = interleave ? 1 : 0;
  int d = 0;
  for (int a = 0; a < ndim; ++a) {
    if (log2_shape[a] < 1 || log2_shape[a] > 30) {
      set_error("qtt_decompose: log2 size %d out of range [1, 30]", log2_shape[a]);
      return QTT_EINVAL;
    }
    desc.log2_shape[a] = log2_shape[a];
    d += log2_shape[a];
  }
  if (d < 2 || d > 30) { set_error("qtt_decompose: total modes d=%d outside [2, 30]", d); return QTT_EINVAL; }
  desc.d = d;
  st = check_trunc(tr, dt, d, true);
  if (st != QTT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  qtt_tensor* t = nullptr;
  std::vector<int> caps = rank_caps(d, tr->rmax, QTT_RANK_CAP);
  if (tr->fixed_ranks) caps.assign(tr->fixed_ranks, tr->fixed_ranks + d + 1);
  st = tensor_alloc(desc, caps, s, &t);
  if (st != QTT_OK) return st;
  const void* v = x;
  void* perm = nullptr;
  if (ndim == 2 && desc.interleave) {
    perm = scratch_alloc(elem_size(dt) << d, s);
    if (!perm) { tensor_free_async(t, s); set_error("qtt_decompose: scratch"); return QTT_ENOMEM; }
    if (dt == QTT_F64)
      launch_morton_gather<double>((const double*)x, (double*)perm, log2_shape[1], log2_shape[0], 1, s);
    else
      launch_morton_gather<float2>((const float2*)x, (float2*)perm, log2_shape[1], log2_shape[0], 1, s);
    v = perm;
  }
  if (dt == QTT_F64) st = tt_svd<double>((const double*)v, d, *tr, t, s);
  else st = tt_svd<float2>((const float2*)v, d, *tr, t, s);
  if (perm) scratch_free(perm, s);
  if (st != QTT_OK) { tensor_free_async(t, s); return st; }
  *out = t;
  return QTT_OK;
}

qtt_status qtt_decompose_rsvd(const void* x, qtt_dtype dt, int log2_len, int rmax, int p,
                              const void* omega, unsigned long long seed, void* stream,
                              qtt_tensor** out) {
  g_err[0] = 0;
  if (!x || !out) { set_error("qtt_decompose_rsvd: NULL argument"); return QTT_EINVAL; }
  Touch tg{(cudaStream_t)stream, nullptr, nullptr, out};
  {
    const qtt_status dst = dtype_status(dt, "qtt_decompose_rsvd");
    if (dst != QTT_OK) return dst;
  }
  if (log2_len < 2 || log2_len > 30) {
    set_error("qtt_decompose_rsvd: log2 length %d outside [2, 30]", log2_len);
    return QTT_EINVAL;
  }
  if (rmax < 1 || rmax > QTT_RANK_CAP || p < 1 || rmax + p > 96) {
    set_error("qtt_decompose_rsvd: need 1 <= rmax <= %d, p >= 1, rmax + p <= 96", QTT_RANK_CAP);
    return QTT_EINVAL;
  }
  TensorDesc desc;
  desc.dt = dt;
  desc.ndim = 1;
  desc.interleave = 0;
  desc.log2_shape[0] = log2_len;
  desc.d = log2_len;
  cudaStream_t s = (cudaStream_t)stream;
  qtt_tensor* t = nullptr;
  qtt_status st = tensor_alloc(desc, rank_caps(log2_len, rmax, QTT_RANK_CAP), s, &t);
  if (st != QTT_OK) return st;
  const qtt_trunc tr{0.0, rmax, 1, 0.0};
  const RsvdOpt rs{p, omega, seed};
  if (dt == QTT_F64) st = tt_svd<double>((const double*)x, log2_len, tr, t, s, &rs);
  else st = tt_svd<float2>((const float2*)x, log2_len, tr, t, s, &rs);
  if (st != QTT_OK) { tensor_free_async(t, s); return st; }
  *out = t;
  return QTT_OK;
}

qtt_status qtt_conv_sinc(const qtt_tensor* f, const double* B, int normalize, double eps_op,
                         const qtt_trunc* round_tr, int sketch, unsigned long long seed,
                         void* stream, qtt_tensor** out) {
  g_err[0] = 0;
  if (!f || !B || !out) { set_error("qtt_conv_sinc: NULL argument"); return QTT_EINVAL; }
  Touch tg{(cudaStream_t)stream, f, nullptr, out};
  qtt_status st = check_trunc(round_tr, f->desc.dt, f->desc.d);
  if (st != QTT_OK) return st;
  if (!(eps_op > 0.0) || eps_op >= 1.0) { set_error("qtt_conv_sinc: eps_op must be in (0, 1)"); return QTT_EINVAL; }
  for (int a = 0; a < f->desc.ndim; ++a)
    if (!(B[a] > 0.0)) { set_error("qtt_conv_sinc: B must be positive"); return QTT_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  if (f->desc.ndim == 1) {
    qtt_op* op = nullptr;
    st = cached_op(f->desc.d, B[0], normalize ? 1 : 0, eps_op, f->desc.dt, s, &op);
    if (st != QTT_OK) return st;
    return round_product(op, f, *round_tr, sketch, seed, s, out);
  }
  qtt_op* ox = nullptr;
  qtt_op* oy = nullptr;
  st = cached_embed(f->desc, 0, B[0], normalize ? 1 : 0, eps_op, s, &ox);
  if (st != QTT_OK) return st;
  st = cached_embed(f->desc, 1, B[1], normalize ? 1 : 0, eps_op, s, &oy);
  if (st != QTT_OK) return st;
  qtt_tensor* y1 = nullptr;
  st = round_product(ox, f, *round_tr, sketch, seed, s, &y1);
  if (st != QTT_OK) return st;
  st = round_product(oy, y1, *round_tr, sketch, seed + 0x9E3779B97F4A7C15ULL, s, out);
  tensor_free_async(y1, s);
  return st;
}

qtt_status qtt_round(qtt_tensor* t, const qtt_trunc* tr, int sketch, unsigned long long seed,
                     void* stream) {
  g_err[0] = 0;
  if (!t) { set_error("qtt_round: NULL tensor"); return QTT_EINVAL; }
  Touch tg{(cudaStream_t)stream, t, nullptr, nullptr};
  qtt_status st = check_trunc(tr, t->desc.dt, t->desc.d);
  if (st != QTT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  qtt_op* id = nullptr;
  st = cached_identity(t->desc.d, t->desc.dt, s, &id);
  if (st != QTT_OK) return st;
  qtt_tensor* y = nullptr;
  st = round_product(id, t, *tr, sketch, seed, s, &y);
  if (st != QTT_OK) return st;
  // move y's storage into t
  scratch_free(t->cores, s);
  t->rcap = y->rcap;
  t->off = y->off;
  t->total = y->total;
  t->cores = y->cores;
  t->ranks = y->ranks;
  t->status = y->status;
  t->norm2 = y->norm2;
  t->margin = y->margin;
  if (y->used) cudaEventDestroy(y->used);
  delete y;
  return QTT_OK;
}

qtt_status qtt_to_full(const qtt_tensor* t, void* y, void* stream) {
  g_err[0] = 0;
  if (!t || !y) { set_error("qtt_to_full: NULL argument"); return QTT_EINVAL; }
  Touch tg{(cudaStream_t)stream, t, nullptr, nullptr};
  cudaStream_t s = (cudaStream_t)stream;
  if (t->desc.dt == QTT_F64) return tt_full<double>(t, (double*)y, s);
  return tt_full<float2>(t, (float2*)y, s);
}

qtt_status qtt_get_margins(const qtt_tensor* t, double* margins_host, void* stream) {
  g_err[0] = 0;
  if (!t || !margins_host) { set_error("qtt_get_margins: NULL argument"); return QTT_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  qtt_status st = cuda_check(cudaMemcpyAsync(margins_host, t->margin,
                                             sizeof(double) * (t->desc.d + 1),
                                             cudaMemcpyDeviceToHost, s), "qtt_get_margins");
  if (st != QTT_OK) return st;
  return cuda_check(cudaStreamSynchronize(s), "qtt_get_margins sync");
}

qtt_status qtt_get_ranks(const qtt_tensor* t, int* ranks_host, void* stream) {
  g_err[0] = 0;
  if (!t || !ranks_host) { set_error("qtt_get_ranks: NULL argument"); return QTT_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  int status = 0;
  qtt_status st = cuda_check(cudaMemcpyAsync(ranks_host, t->ranks, sizeof(int) * (t->desc.d + 1),
                                             cudaMemcpyDeviceToHost, s), "qtt_get_ranks");
  if (st != QTT_OK) return st;
  st = cuda_check(cudaMemcpyAsync(&status, t->status, sizeof(int), cudaMemcpyDeviceToHost, s),
                  "qtt_get_ranks status");
  if (st != QTT_OK) return st;
  st = cuda_check(cudaStreamSynchronize(s), "qtt_get_ranks sync");
  if (st != QTT_OK) return st;
  if (status & DEV_ST_JACOBI_LIMIT) {
    set_error("a Jacobi eigen-solve reached its sweep limit before convergence");
    return QTT_ETIMEOUT;
  }
  if (status & DEV_ST_RANK_OVERFLOW) { set_error("a rank exceeded its capacity"); return QTT_ERANK; }
  if (status & DEV_ST_NONFINITE) {
    set_error("an eigen-solve met a non-finite value (NaN or Inf in the data)");
    return QTT_ENUMERIC;
  }
  return QTT_OK;
}

qtt_status qtt_get_info(const qtt_tensor* t, int* d, qtt_dtype* dt, int* ndim, int* log2_shape,
                        int* interleave) {
  if (!t) { set_error("qtt_get_info: NULL tensor"); return QTT_EINVAL; }
  if (d) *d = t->desc.d;
  if (dt) *dt = t->desc.dt;
  if (ndim) *ndim = t->desc.ndim;
  if (log2_shape) {
    log2_shape[0] = t->desc.log2_shape[0];
    if (t->desc.ndim == 2) log2_shape[1] = t->desc.log2_shape[1];
  }
  if (interleave) *interleave = t->desc.interleave;
  return QTT_OK;
}

qtt_status qtt_get_cores(const qtt_tensor* t, void* host_buf, void* stream) {
  g_err[0] = 0;
  if (!t || !host_buf) { set_error("qtt_get_cores: NULL argument"); return QTT_EINVAL; }
  const int d = t->desc.d;
  std::vector<int> r(d + 1);
  qtt_status st = qtt_get_ranks(t, r.data(), stream);
  if (st != QTT_OK && st != QTT_ETIMEOUT) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t esz = elem_size(t->desc.dt);
  char* dst = (char*)host_buf;
  for (int k = 0; k < d; ++k) {
    const size_t cnt = (size_t)r[k] * 2 * r[k + 1];
    st = cuda_check(cudaMemcpyAsync(dst, (const char*)t->cores + esz * t->off[k], esz * cnt,
                                    cudaMemcpyDeviceToHost, s), "qtt_get_cores");
    if (st != QTT_OK) return st;
    dst += esz * cnt;
  }
  return cuda_check(cudaStreamSynchronize(s), "qtt_get_cores sync");
}

qtt_status qtt_from_cores(const void* host_cores, const int* ranks, int d, qtt_dtype dt, int ndim,
                          const int* log2_shape, int interleave, void* stream, qtt_tensor** out) {
  g_err[0] = 0;
  if (!host_cores || !ranks || !log2_shape || !out) { set_error("qtt_from_cores: NULL argument"); return QTT_EINVAL; }
  Touch tg{(cudaStream_t)stream, nullptr, nullptr, out};
  if (dt == QTT_F32 || dt == QTT_C128) return dtype_status(dt, "qtt_from_cores");
  if (!valid_dtype(dt) || d < 2 || d > 30 || (ndim != 1 && ndim != 2)) {
    set_error("qtt_from_cores: bad dtype/d/ndim");
    return QTT_EINVAL;
  }
  if (ranks[0] != 1 || ranks[d] != 1) { set_error("qtt_from_cores: boundary ranks must be 1"); return QTT_EINVAL; }
  int dsum = 0;
  for (int a = 0; a < ndim; ++a) dsum += log2_shape[a];
  if (dsum != d) { set_error("qtt_from_cores: log2 shape does not add up to d"); return QTT_EINVAL; }
  for (int k = 1; k < d; ++k)
    if (ranks[k] < 1 || ranks[k] > QTT_PRODUCT_CAP) { set_error("qtt_from_cores: rank %d out of range", ranks[k]); return QTT_EINVAL; }
  TensorDesc desc;
  desc.d = d;
  desc.dt = dt;
  desc.ndim = ndim;
  desc.interleave = interleave ? 1 : 0;
  for (int a = 0; a < ndim; ++a) desc.log2_shape[a] = log2_shape[a];
  std::vector<int> rc(ranks, ranks + d + 1);
  cudaStream_t s = (cudaStream_t)stream;
  qtt_tensor* t = nullptr;
  qtt_status st = tensor_alloc(desc, rc, s, &t);
  if (st != QTT_OK) return st;
  st = cuda_check(cudaMemcpyAsync(t->cores, host_cores, elem_size(dt) * t->total,
                                  cudaMemcpyHostToDevice, s), "qtt_from_cores");
  if (st != QTT_OK) { tensor_free_async(t, s); return st; }
  set_ranks_from_host(t->ranks, rc, s);
  st = cuda_check(cudaStreamSynchronize(s), "qtt_from_cores sync");
  if (st != QTT_OK) { tensor_free_async(t, s); return st; }
  *out = t;
  return QTT_OK;
}

void qtt_free(qtt_tensor* t) {
  if (!t) return;
  cudaStream_t fs = t->used ? free_stream() : nullptr;
  if (fs) {
    // released in stream order after the last call that used the handle
    cudaStreamWaitEvent(fs, t->used, 0);
    tensor_free_async(t, fs);
    return;
  }
  if (t->cores) {
    cudaDeviceSynchronize();
    cudaFree(t->cores);
  }
  if (t->used) cudaEventDestroy(t->used);
  delete t;
}

void qtt_free_async(qtt_tensor* t, void* stream) { tensor_free_async(t, (cudaStream_t)stream); }

qtt_status qtt_op_create(int d, double B, int normalize, double eps_op, qtt_dtype dt, void* stream,
                         qtt_op** out) {
  g_err[0] = 0;
  if (dt == QTT_F32 || dt == QTT_C128) return dtype_status(dt, "qtt_op_create");
  if (!out || !valid_dtype(dt)) { set_error("qtt_op_create: bad argument"); return QTT_EINVAL; }
  if (!(B > 0.0) || !(eps_op > 0.0) || eps_op >= 1.0) { set_error("qtt_op_create: B > 0 and eps_op in (0,1) required"); return QTT_EINVAL; }
  return op_sinc_create(d, B, normalize ? 1 : 0, eps_op, dt, (cudaStream_t)stream, out);
}

qtt_status qtt_op_get_ranks(const qtt_op* op, int* ranks_host) {
  if (!op || !ranks_host) { set_error("qtt_op_get_ranks: NULL argument"); return QTT_EINVAL; }
  for (int k = 0; k <= op->d; ++k) ranks_host[k] = op->P[k];
  return QTT_OK;
}

qtt_status qtt_op_get_cores(const qtt_op* op, void* host_buf) {
  if (!op || !host_buf) { set_error("qtt_op_get_cores: NULL argument"); return QTT_EINVAL; }
  const size_t rsz = op->dt == QTT_F64 ? sizeof(double) : sizeof(float);
  return cuda_check(cudaMemcpy(host_buf, op->cores, rsz * op->total, cudaMemcpyDeviceToHost),
                    "qtt_op_get_cores");
}

void qtt_op_free(qtt_op* op) {
  if (!op) return;
  cudaDeviceSynchronize();
  op_free(op);
}

qtt_status qtt_matvec(const qtt_op* op, const qtt_tensor* x, void* stream, qtt_tensor** out) {
  g_err[0] = 0;
  if (!op || !x || !out) { set_error("qtt_matvec: NULL argument"); return QTT_EINVAL; }
  Touch tg{(cudaStream_t)stream, x, nullptr, out};
  return matvec(op, x, (cudaStream_t)stream, out);
}

qtt_status qtt_sinc_padded(int log2_n, long long N, double B, int normalize, qtt_dtype dt,
                           void* g_dev, void* stream) {
  g_err[0] = 0;
  if (!g_dev) { set_error("qtt_sinc_padded: NULL output"); return QTT_EINVAL; }
  if (dt == QTT_F32 || dt == QTT_C128) return dtype_status(dt, "qtt_sinc_padded");
  if (!valid_dtype(dt) || log2_n < 1 || log2_n > 30) {
    set_error("qtt_sinc_padded: bad dtype or log2_n");
    return QTT_EINVAL;
  }
  const long long n = 1LL << log2_n;
  if (N < 1 || N % 2 == 0 || 2 * N - 1 > n) {
    set_error("qtt_sinc_padded: need N odd with 2N - 1 <= 2^log2_n (got N = %lld)", N);
    return QTT_EINVAL;
  }
  return sinc_padded(log2_n, N, B, normalize, dt, g_dev, (cudaStream_t)stream);
}

qtt_status qtt_fft(const qtt_tensor* x, int inverse, const qtt_trunc* tr, int sketch,
                   unsigned long long seed, void* stream, qtt_tensor** out) {
  g_err[0] = 0;
  if (!x || !out) { set_error("qtt_fft: NULL argument"); return QTT_EINVAL; }
  RepairScope rs;
  Touch tg{(cudaStream_t)stream, x, nullptr, out};
  qtt_trunc t0 = {0.0, 0, 1, 0.0, QTT_PREC_AUTO, nullptr};
  if (tr) {
    qtt_status st = check_trunc(tr, x->desc.dt, x->desc.d);
    if (st != QTT_OK) return st;
    t0 = *tr;
  }
  cudaStream_t s = (cudaStream_t)stream;
  qtt_op* id = nullptr;
  qtt_status st = cached_identity(x->desc.d, x->desc.dt, s, &id);
  if (st != QTT_OK) return st;
  return fft_transform(x, inverse, t0, id, sketch, seed, s, out);
}

// diagnostics: hand the memory pool a block filled with one byte value, so
// that the library's next scratch allocations start from known contents
qtt_status qtt_debug_fill_pool(size_t bytes, int value, void* stream) {
  g_err[0] = 0;
  cudaStream_t s = (cudaStream_t)stream;
  void* p = scratch_alloc(bytes, s);
  if (!p) { set_error("qtt_debug_fill_pool: allocation of %zu bytes failed", bytes); return QTT_ENOMEM; }
  cudaMemsetAsync(p, value & 0xff, bytes, s);
  scratch_free(p, s);
  return cuda_check(cudaStreamSynchronize(s), "qtt_debug_fill_pool");
}

void qtt_release_workspace(void) {
  cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lk(g_cache_mu);
  for (auto& kv : g_op_cache) op_free(kv.second);
  for (auto& kv : g_emb_cache) op_free(kv.second);
  for (auto& kv : g_id_cache) op_free(kv.second);
  for (auto& kv : g_tr_cache) op_free(kv.second);
  g_tr_cache.clear();
  sketch_cache_clear();
  g_op_cache.clear();
  g_emb_cache.clear();
  g_id_cache.clear();
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
  }
}

static bool same_layout(const qtt_tensor* a, const qtt_tensor* b) {
  if (a->desc.d != b->desc.d || a->desc.dt != b->desc.dt || a->desc.ndim != b->desc.ndim) return false;
  for (int i = 0; i < a->desc.ndim; ++i)
    if (a->desc.log2_shape[i] != b->desc.log2_shape[i]) return false;
  return a->desc.ndim == 1 || a->desc.interleave == b->desc.interleave;
}

qtt_status qtt_conv_adjoint(const qtt_tensor* f, const qtt_tensor* r, const double* B,
                            int normalize, double eps_op, const qtt_trunc* round_tr, int sketch,
                            unsigned long long seed, void* const* grad_cores,
                            qtt_tensor** adj_out, void* stream) {
  g_err[0] = 0;
  if (!r || !B) { set_error("qtt_conv_adjoint: NULL argument"); return QTT_EINVAL; }
  Touch tg{(cudaStream_t)stream, f, r, adj_out};
  if (grad_cores && !f) { set_error("qtt_conv_adjoint: gradients need f"); return QTT_EINVAL; }
  if (f && !same_layout(f, r)) { set_error("qtt_conv_adjoint: f and r differ in shape or type"); return QTT_EINVAL; }
  if (grad_cores)
    for (int k = 0; k < r->desc.d; ++k)
      if (!grad_cores[k]) { set_error("qtt_conv_adjoint: grad_cores[%d] is NULL", k); return QTT_EINVAL; }
  qtt_status st = check_trunc(round_tr, r->desc.dt, r->desc.d);
  if (st != QTT_OK) return st;
  if (!(eps_op > 0.0) || eps_op >= 1.0) { set_error("qtt_conv_adjoint: eps_op must be in (0, 1)"); return QTT_EINVAL; }
  for (int a = 0; a < r->desc.ndim; ++a)
    if (!(B[a] > 0.0)) { set_error("qtt_conv_adjoint: B must be positive"); return QTT_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  const int nrm = normalize ? 1 : 0;
  qtt_tensor* adj = nullptr;
  if (r->desc.ndim == 1) {
    qtt_op* op = nullptr;
    qtt_op* opT = nullptr;
    st = cached_op(r->desc.d, B[0], nrm, eps_op, r->desc.dt, s, &op);
    if (st == QTT_OK) st = cached_transpose(op, s, &opT);
    if (st == QTT_OK) st = round_product(opT, r, *round_tr, sketch, seed, s, &adj);
  } else {
    // (T_y T_x)^H = T_x^H T_y^H: the y adjoint first
    qtt_op *ox = nullptr, *oy = nullptr, *oxT = nullptr, *oyT = nullptr;
    st = cached_embed(r->desc, 0, B[0], nrm, eps_op, s, &ox);
    if (st == QTT_OK) st = cached_embed(r->desc, 1, B[1], nrm, eps_op, s, &oy);
    if (st == QTT_OK) st = cached_transpose(ox, s, &oxT);
    if (st == QTT_OK) st = cached_transpose(oy, s, &oyT);
    qtt_tensor* a1 = nullptr;
    if (st == QTT_OK) st = round_product(oyT, r, *round_tr, sketch, seed, s, &a1);
    if (st == QTT_OK) {
      st = round_product(oxT, a1, *round_tr, sketch, seed + 0x9E3779B97F4A7C15ULL, s, &adj);
      tensor_free_async(a1, s);
    }
  }
  if (st != QTT_OK) return st;
  if (grad_cores) {
    st = env_sweep(f, adj, 2.0, 0.0, grad_cores, nullptr, s);
    if (st != QTT_OK) { tensor_free_async(adj, s); return st; }
  }
  if (adj_out) *adj_out = adj;
  else tensor_free_async(adj, s);
  return QTT_OK;
}

qtt_status qtt_core_grads(const qtt_tensor* f, const qtt_tensor* w, double alpha, double beta,
                          void* const* grad_cores, void* stream) {
  g_err[0] = 0;
  if (!f || !w || !grad_cores) { set_error("qtt_core_grads: NULL argument"); return QTT_EINVAL; }
  Touch tg{(cudaStream_t)stream, f, w, nullptr};
  if (!same_layout(f, w)) { set_error("qtt_core_grads: f and w differ in shape or type"); return QTT_EINVAL; }
  for (int k = 0; k < f->desc.d; ++k)
    if (!grad_cores[k]) { set_error("qtt_core_grads: grad_cores[%d] is NULL", k); return QTT_EINVAL; }
  return env_sweep(f, w, alpha, beta, grad_cores, nullptr, (cudaStream_t)stream);
}

qtt_status qtt_dot(const qtt_tensor* x, const qtt_tensor* y, double* out_dev, void* stream) {
  g_err[0] = 0;
  if (!x || !y || !out_dev) { set_error("qtt_dot: NULL argument"); return QTT_EINVAL; }
  Touch tg{(cudaStream_t)stream, x, y, nullptr};
  if (!same_layout(x, y)) { set_error("qtt_dot: tensors differ in shape or type"); return QTT_EINVAL; }
  return env_sweep(x, y, 0.0, 0.0, nullptr, (double2*)out_dev, (cudaStream_t)stream);
}

qtt_status qtt_add(double alpha, const qtt_tensor* x, double beta, const qtt_tensor* y,
                   void* stream, qtt_tensor** out) {
  g_err[0] = 0;
  if (!x || !y || !out) { set_error("qtt_add: NULL argument"); return QTT_EINVAL; }
  Touch tg{(cudaStream_t)stream, x, y, out};
  if (!same_layout(x, y)) { set_error("qtt_add: tensors differ in shape or type"); return QTT_EINVAL; }
  return tt_add(alpha, x, beta, y, (cudaStream_t)stream, out);
}

qtt_status qtt_hadamard(const qtt_tensor* x, const qtt_tensor* y, void* stream, qtt_tensor** out) {
  g_err[0] = 0;
  if (!x || !y || !out) { set_error("qtt_hadamard: NULL argument"); return QTT_EINVAL; }
  RepairScope rs;
  Touch tg{(cudaStream_t)stream, x, y, out};
  if (!same_layout(x, y)) { set_error("qtt_hadamard: tensors differ in shape or type"); return QTT_EINVAL; }
  return hadamard(x, y, (cudaStream_t)stream, out);
}

qtt_status qtt_from_device_cores(const void* const* cores, const int* ranks, int d, qtt_dtype dt,
                                 int ndim, const int* log2_shape, int interleave, void* stream,
                                 qtt_tensor** out) {
  g_err[0] = 0;
  if (!cores || !ranks || !log2_shape || !out) { set_error("qtt_from_device_cores: NULL argument"); return QTT_EINVAL; }
  Touch tg{(cudaStream_t)stream, nullptr, nullptr, out};
  if (dt == QTT_F32 || dt == QTT_C128) return dtype_status(dt, "qtt_from_device_cores");
  if (!valid_dtype(dt) || d < 2 || d > 30 || (ndim != 1 && ndim != 2)) {
    set_error("qtt_from_device_cores: bad dtype/d/ndim");
    return QTT_EINVAL;
  }
  if (ranks[0] != 1 || ranks[d] != 1) { set_error("qtt_from_device_cores: boundary ranks must be 1"); return QTT_EINVAL; }
  int dsum = 0;
  for (int a = 0; a < ndim; ++a) dsum += log2_shape[a];
  if (dsum != d) { set_error("qtt_from_device_cores: log2 shape does not add up to d"); return QTT_EINVAL; }
  for (int k = 1; k < d; ++k)
    if (ranks[k] < 1 || ranks[k] > QTT_PRODUCT_CAP) { set_error("qtt_from_device_cores: rank %d out of range", ranks[k]); return QTT_EINVAL; }
  for (int k = 0; k < d; ++k)
    if (!cores[k]) { set_error("qtt_from_device_cores: cores[%d] is NULL", k); return QTT_EINVAL; }
  TensorDesc desc;
  desc.d = d;
  desc.dt = dt;
  desc.ndim = ndim;
  desc.interleave = interleave ? 1 : 0;
  for (int a = 0; a < ndim; ++a) desc.log2_shape[a] = log2_shape[a];
  std::vector<int> rc(ranks, ranks + d + 1);
  cudaStream_t s = (cudaStream_t)stream;
  qtt_tensor* t = nullptr;
  qtt_status st = tensor_alloc(desc, rc, s, &t);
  if (st != QTT_OK) return st;
  const size_t esz = elem_size(dt);
  for (int k = 0; k < d; ++k) {
    st = cuda_check(cudaMemcpyAsync((char*)t->cores + esz * t->off[k], cores[k],
                                    esz * (size_t)rc[k] * 2 * rc[k + 1], cudaMemcpyDeviceToDevice, s),
                    "qtt_from_device_cores");
    if (st != QTT_OK) { tensor_free_async(t, s); return st; }
  }
  set_ranks_from_host(t->ranks, rc, s);
  *out = t;
  return QTT_OK;
}

}  // extern "C"
