// Internal declarations of libqtt (not part of the C ABI).
//
// Element types: T = double (real, FP64 path) or float2 (complex float, FP32
// path).  R is the matching real type.  Reductions that feed rank decisions
// (traces, partial-Gram sums) are carried in double.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <vector>
#include <string>
#include <atomic>
#include "../../include/qtt.h"

namespace qtt {

// ---------------------------------------------------------------- scalars
template <typename T> struct Sc;
template <> struct Sc<double> {
  using R = double;
  static constexpr bool cplx = false;
  static constexpr double eps = 2.220446049250313e-16;
};
template <> struct Sc<float2> {
  using R = float;
  static constexpr bool cplx = true;
  static constexpr double eps = 1.1920928955078125e-07;
};

__host__ __device__ __forceinline__ double zero_of(double) { return 0.0; }
__host__ __device__ __forceinline__ float2 zero_of(float2) { return make_float2(0.f, 0.f); }
template <typename T> __host__ __device__ __forceinline__ T szero() { return zero_of(T()); }
__host__ __device__ __forceinline__ double sone(double) { return 1.0; }
__host__ __device__ __forceinline__ float2 sone(float2) { return make_float2(1.f, 0.f); }

__host__ __device__ __forceinline__ double conjg(double a) { return a; }
__host__ __device__ __forceinline__ float2 conjg(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double sadd(double a, double b) { return a + b; }
__host__ __device__ __forceinline__ float2 sadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double ssub(double a, double b) { return a - b; }
__host__ __device__ __forceinline__ float2 ssub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double smul(double a, double b) { return a * b; }
__host__ __device__ __forceinline__ float2 smul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// real scaling
__host__ __device__ __forceinline__ double rscale(double a, double s) { return a * s; }
__host__ __device__ __forceinline__ float2 rscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double sreal(double a) { return a; }
__host__ __device__ __forceinline__ float sreal(float2 a) { return a.x; }
__host__ __device__ __forceinline__ double simag(double) { return 0.0; }
__host__ __device__ __forceinline__ float simag(float2 a) { return a.y; }
template <typename T> __host__ __device__ __forceinline__ T make_scalar(typename Sc<T>::R re, typename Sc<T>::R im);
template <> __host__ __device__ __forceinline__ double make_scalar<double>(double re, double) { return re; }
template <> __host__ __device__ __forceinline__ float2 make_scalar<float2>(float re, float im) { return make_float2(re, im); }
__host__ __device__ __forceinline__ double rmax(double a, double b) { return fmax(a, b); }
__host__ __device__ __forceinline__ float rmax(float a, float b) { return fmaxf(a, b); }
__host__ __device__ __forceinline__ double rabs(double a) { return fabs(a); }
__host__ __device__ __forceinline__ float rabs(float a) { return fabsf(a); }
__host__ __device__ __forceinline__ double sabs2(double a) { return a * a; }
__host__ __device__ __forceinline__ float sabs2(float2 a) { return a.x * a.x + a.y * a.y; }

// acc += a * b
__device__ __forceinline__ void mac(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void mac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void macc(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void macc(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}
// acc += a * conj(b)
__device__ __forceinline__ void macb(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void macb(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.y, b.x, acc.y);
  acc.y = fmaf(-a.x, b.y, acc.y);
}
// acc += r * b  (r real)
__device__ __forceinline__ void rmac(double& acc, double r, double b) { acc = fma(r, b, acc); }
__device__ __forceinline__ void rmac(float2& acc, float r, float2 b) {
  acc.x = fmaf(r, b.x, acc.x);
  acc.y = fmaf(r, b.y, acc.y);
}
// acc += r * b  (r complex)
__device__ __forceinline__ void rmac(float2& acc, float2 r, float2 b) {
  acc.x = fmaf(r.x, b.x, acc.x);
  acc.x = fmaf(-r.y, b.y, acc.x);
  acc.y = fmaf(r.x, b.y, acc.y);
  acc.y = fmaf(r.y, b.x, acc.y);
}

// Warp-wide sum of a T value with float shuffles for the FP32 path.
__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ float2 warp_sum(float2 v) {
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  return v;
}
// one shuffle of a T value (full-warp mask; all lanes must take part)
__device__ __forceinline__ double shfl_xor_s(double v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ float2 shfl_xor_s(float2 v, int off) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, off), __shfl_xor_sync(0xffffffffu, v.y, off));
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Compensated (Kahan) accumulation for the FP32 path: acc + comp carries the
// sum of rounded products to ~1 ulp instead of ~sqrt(K) ulp.  FP64 sums are
// plain.
struct KAcc64 {
  double s = 0.0;
  __device__ __forceinline__ void add_mul(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ void add_cmul(double a, double b) { s = fma(a, b, s); }   // conj(a) b
  __device__ __forceinline__ void add_rmul(double r, double b) { s = fma(r, b, s); }
  __device__ __forceinline__ double get() const { return s; }
};
struct KAcc32 {
  float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
  __device__ __forceinline__ void add(float2 p) {
    float y = p.x - c.x, t = s.x + y;
    c.x = (t - s.x) - y;
    s.x = t;
    y = p.y - c.y;
    t = s.y + y;
    c.y = (t - s.y) - y;
    s.y = t;
  }
  __device__ __forceinline__ void add_mul(float2 a, float2 b) {
    add(make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)));
  }
  __device__ __forceinline__ void add_cmul(float2 a, float2 b) {   // conj(a) b
    add(make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x)));
  }
  __device__ __forceinline__ void add_rmul(float r, float2 b) { add(make_float2(r * b.x, r * b.y)); }
  __device__ __forceinline__ float2 get() const { return make_float2(s.x - c.x, s.y - c.y); }
};
// Dot2 accumulation (Ogita, Rump and Oishi, "Accurate sum and dot
// product", 2005): each product is split exactly into p + e by an FMA and
// the running sum is carried by TwoSum with the rounding errors collected in
// c, so the result is as accurate as a sum in twice the working precision:
// its error is about eps |result| + eps^2 sum |a b|.  Used where FP32 sums
// cancel strongly (projections onto nearly orthogonal directions).
struct Dot2Acc32 {
  float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
  __device__ __forceinline__ static void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
  }
  __device__ __forceinline__ void add_term(float& sm, float& cm, float p, float e) {
    float q;
    two_sum(sm, p, sm, q);
    cm += q + e;
  }
  // acc += a * b (complex)
  __device__ __forceinline__ void add_mul(float2 a, float2 b) {
    const float p1 = a.x * b.x, e1 = fmaf(a.x, b.x, -p1);
    const float p2 = -a.y * b.y, e2 = fmaf(-a.y, b.y, -p2);
    const float p3 = a.x * b.y, e3 = fmaf(a.x, b.y, -p3);
    const float p4 = a.y * b.x, e4 = fmaf(a.y, b.x, -p4);
    add_term(s.x, c.x, p1, e1);
    add_term(s.x, c.x, p2, e2);
    add_term(s.y, c.y, p3, e3);
    add_term(s.y, c.y, p4, e4);
  }
  __device__ __forceinline__ float2 get() const { return make_float2(s.x + c.x, s.y + c.y); }
};
template <typename T> struct Dot2Of;
template <> struct Dot2Of<double> { using type = KAcc64; };
template <> struct Dot2Of<float2> { using type = Dot2Acc32; };

template <typename T> struct KAccOf;
template <> struct KAccOf<double> { using type = KAcc64; };
template <> struct KAccOf<float2> { using type = KAcc32; };

// double-precision accumulator of a T value (for reductions)
__host__ __device__ __forceinline__ double2 to_d2(double a) { return make_double2(a, 0.0); }
__host__ __device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ void from_d2(double2 v, double& o) { o = v.x; }
__host__ __device__ __forceinline__ void from_d2(double2 v, float2& o) { o = make_float2((float)v.x, (float)v.y); }

// ---------------------------------------------------------------- status
// Device status word bits (OR-ed by kernels; read by qtt_get_ranks).
enum : int {
  DEV_ST_JACOBI_LIMIT = 1,   // Jacobi sweep limit reached before convergence
  DEV_ST_RANK_OVERFLOW = 2,  // a rank larger than its capacity was requested
  DEV_ST_NONFINITE = 4,      // an eigen-solve met a non-finite value (NaN / Inf input)
};

// ---------------------------------------------------------------- handles
struct TensorDesc {
  int d = 0;
  qtt_dtype dt = QTT_C64;
  int ndim = 1;
  int log2_shape[2] = {0, 0};   // {d} or {dy, dx}
  int interleave = 1;
};

}  // namespace qtt

struct qtt_tensor {
  qtt::TensorDesc desc;
  std::vector<int> rcap;          // host capacity per cut, d+1 entries
  std::vector<size_t> off;        // element offset of core k (0-based), d entries
  size_t total = 0;               // elements allocated for cores
  void* cores = nullptr;          // device, element type of desc.dt
  int* ranks = nullptr;           // device, d+1 ints
  int* status = nullptr;          // device, 1 int
  double* norm2 = nullptr;        // device, 1 double (squared norm at creation)
  double* margin = nullptr;       // device, d+1 doubles: eps-rule decision margin per cut (NaN: none)
  cudaEvent_t used = nullptr;     // recorded on the stream of every call that used the handle
};

struct qtt_op {
  int d = 0;                      // number of modes the operator acts on
  qtt_dtype dt = QTT_C64;         // data type it is applied to (cores are real R)
  int cplx = 0;                   // 1: complex cores (float2, QTT_C64 only; the QTT-FFT stages)
  std::vector<int> P;             // ranks P_0..P_d (host)
  std::vector<size_t> off;        // offsets of the cores (elements of R)
  size_t total = 0;
  void* cores = nullptr;          // device, real (double for F64, float for C64)
};

namespace qtt {

size_t elem_size(qtt_dtype dt);
void set_error(const char* fmt, ...);
void clear_error();   // empty the thread-local message (start of an entry point)
qtt_status cuda_check(cudaError_t e, const char* what);

// capacities: r_k <= min(2^k, 2^(d-k), rmax, cap)
std::vector<int> rank_caps(int d, int rmax, int cap);

// allocate a tensor handle with the given capacity profile (no data)
qtt_status tensor_alloc(const TensorDesc& desc, const std::vector<int>& rcap,
                        cudaStream_t s, qtt_tensor** out);

// ------------------------------------------------------------- TT-SVD
// Decompose the vector v (2^d elements, QTT order, device) into t (allocated
// by the caller with caps from rank_caps).  eps/rmax/refine as qtt_trunc.
// Max rank TT-RSVD (Sec. 5 modification (2)): p > 0 replaces the SVD of
// every unfolding with min(m_k, n_k) > rmax + p by the randomized SVD with
// oversampling p; omega = the Gaussian blocks (see qtt_decompose_rsvd) or
// NULL to draw them on the device from seed.
struct RsvdOpt {
  int p;
  const void* omega;
  unsigned long long seed;
};
template <typename T>
qtt_status tt_svd(const T* v, int d, const qtt_trunc& tr, qtt_tensor* t, cudaStream_t s,
                  const RsvdOpt* rs = nullptr);
// N(0, 1) draws, out[e] for e < n: Philox4x32-10 counter (e, tag), key seed, Box-Muller
void launch_gauss_fill(float* out, long long n, unsigned long long seed, uint32_t tag, cudaStream_t s);
void launch_gauss_fill(double* out, long long n, unsigned long long seed, uint32_t tag, cudaStream_t s);

// ------------------------------------------------------------- small SVD
// One-CTA SVD helper used by the rounding sweeps: see k_svd.cu.
template <typename T>
void launch_gram_eig(const T* gram_part, int nparts, int ldp, const int* mg_ptr, int mg_mul,
                     int mg_cap, int mode, double eps, int dmodes, int rmax, const int* ncols_ptr,
                     int ncols_mul, long long ncols_const, const T* U1, T* Uout, T* core_out,
                     int* rank_out, double* sig_out, double* norm2, int write_norm2,
                     int* status, cudaStream_t s, int relative = 0, double delta = 0.0,
                     int sweeps = -1, double* margin_out = nullptr);

// ------------------------------------------------------------- eigen
enum { EIG_MODE_ALL = 0, EIG_MODE_DECIDE = 1 };

template <typename T>
struct EigArgs {
  const double2* G;     // dense, ld = ldp
  int ldp;
  const int* mg_ptr;    // mg = mg_mul * *mg_ptr, or mg_const when mg_ptr is null
  int mg_mul;
  int mg_const;
  int mode;
  double eps;           // relative accuracy for the rank decision
  int dmodes;           // d (number of modes) for tau = eps / sqrt(d-1) * ||A||
  int rmax;             // cap (> 0)
  const int* ncols_ptr; // ncols = ncols_mul * *ncols_ptr, or ncols_const if null
  int ncols_mul;
  long long ncols_const;
  const T* U1;          // optional: core = U1 * U[:, :r] (U1 is mg x mg, ld mg)
  T* Uout;              // sorted eigenvectors (ld = mg): all (MODE_ALL) or first r
  T* core_out;          // optional: core (ld = mg, r columns)
  int* rank_out;        // MODE_DECIDE: receives r
  double* sig_out;      // optional: sorted eigenvalues
  double* norm2;        // squared norm (read for tau; written when write_norm2)
  int write_norm2;
  int* status;
  int relative;         // 1: small eigenvalues needed to relative accuracy (Jacobi)
  double delta;         // > 0: SV drop-off rank rule instead of eps (MODE_DECIDE)
  int max_sweeps;       // Jacobi sweep limit (0: the default, flagged when reached)
  long long* phase_clk; // optional: clock64() at phase boundaries (diagnostics)
  float ortol_rel;      // tridiagonal solver: cluster gap / ||T|| for Gram-Schmidt
  int ns_steps;         // tridiagonal solver: Newton-Schulz steps
  double* margin_out;   // optional (MODE_DECIDE): margin of the eps-rule decision
  int* orth_flag;       // optional (tridiagonal solver, n <= 32): set to 1 when its
                        // eigenvectors leave max |Z^T Z - I| above 1e-4
  const int* only_if;   // optional (Jacobi solver): run only when *only_if != 0
};

// Margin of an eps-rule rank decision: min over the two tails around the
// cut of |sqrt(tail) - tau| / tau, with tail(r) = sum_{i >= r} lambda_i the
// kept tail and tail(r-1) the one that was too large; NaN when the rank
// was not decided by the eps rule (eps = 0, the drop-off rule, or the cap).
__host__ __device__ inline double rank_margin(double tau2, double tail_kept, double tail_next,
                                              bool has_next) {
  const double tau = sqrt(tau2);
  double m = fabs(sqrt(tail_kept > 0.0 ? tail_kept : 0.0) - tau) / tau;
  if (has_next) {
    const double m2 = fabs(sqrt(tail_next > 0.0 ? tail_next : 0.0) - tau) / tau;
    m = m2 < m ? m2 : m;
  }
  return m;
}


// one-CTA Hermitian eigensolvers (k_svd.cu: Jacobi; k_heev.cu: Householder
// tridiagonalisation + bisection + twisted factorisation, FP32 path)
void launch_heev_tri(const EigArgs<float2>& a, int mg_cap, cudaStream_t s);
void heev_set_cluster_params(double ortol_rel, int ns_steps);
size_t heev_tri_smem_bytes(int mg_cap);

// eigen-decomposition of a dense double2 Gram (k_svd.cu); relative = 1 asks
// for small eigenvalues to relative accuracy (Jacobi)
template <typename T>
void launch_eig_dense(const double2* G, int ldp, const int* mg_ptr, int mg_mul, int mg_const,
                      int mg_cap, int mode, double eps, int dmodes, int rmax,
                      const int* ncols_ptr, int ncols_mul, long long ncols_const, const T* U1,
                      T* Uout, T* core_out, int* rank_out, double* sig_out, double* norm2,
                      int write_norm2, int* status, cudaStream_t s, int relative = 0,
                      double delta = 0.0, int sweeps = -1, double* margin_out = nullptr);

// ------------------------------------------------------------- large ranks
// First call for the current device with this flag word: true once per
// device (per-device one-time set-up such as kernel attributes).
bool first_on_device(std::atomic<unsigned long long>* flags);
// multiprocessors of the current device (grid sizing)
int device_sm_count();

// Blocked Householder QR (k_dense.cu): A (m x n, ld m, m <= 768) is
// overwritten by R and the reflectors; Q (m x nq, ld m) receives the first
// nq columns of the Q factor.  Tm: workspace of big_qr_tm_elems(n) elements.
template <typename T>
qtt_status big_qr_q(T* A, int m, int n, int nq, T* Q, T* Tm, cudaStream_t s);
size_t big_qr_tm_elems(int n);
// A (m x n, ld m) = S^H for S (n x m, ld ls)
template <typename T>
void launch_conj_transpose(const T* S, int ls, int n, int m, T* A, cudaStream_t s);

// C = op(A) B (complex64 B, C; A complex64 or real float), strided and
// batched: batch z = b1 + nb1 b2 offsets every operand by b1 bX1 + b2 bX2.
// Element (i, k) of A at i sAi + k sAk (conjugated when conjA), (k, j) of B at
// k sBk + j sBj, (i, j) of C at i sCi + j sCj.  Fast paths: sAi == 1 or
// sAk == 1, sBk == 1.  Chunks of 16 terms are added with compensation.
template <typename TA>
struct CGemmArgs {
  const TA* A = nullptr;
  long long sAi = 1, sAk = 1, bA1 = 0, bA2 = 0;
  const float2* B = nullptr;
  long long sBk = 1, sBj = 1, bB1 = 0, bB2 = 0;
  float2* C = nullptr;
  long long sCi = 1, sCj = 1, bC1 = 0, bC2 = 0;
  int M = 0, N = 0, K = 0, nb1 = 1, conjA = 0;
};
template <typename TA>
qtt_status cgemm(const CGemmArgs<TA>& g, int nbatch, cudaStream_t s, const char* name);
// C[i + M j] (then to C at sCi, sCj) = compensated sum over s of part[s ldpart + i + M j]
void cgemm_reduce(const float2* part, int splits, long long ldpart, int M, int N, float2* C,
                  long long sCi, long long sCj, cudaStream_t s);
// the same product on the tensor cores (tcgen05, 3xTF32, FP32 accumulators);
// a wait that runs out writes QTT_ETIMEOUT to *status (a device word) if it
// holds QTT_OK
template <typename TA>
qtt_status tc_cgemm(const CGemmArgs<TA>& g, int nbatch, int* status, cudaStream_t s,
                    const char* name);
int tc_gemm_enabled();
// this host thread's small FP32 eigen-solves check their orthonormality and
// repair failed solves (set by the QTT-FFT route's entry points)
void set_heev_repair(int on);
// tile settings of this host thread's Gram passes (0, 0: the defaults)
void set_gram_tiles(int parts_per_sm, int chunk_div);
// per-CTA partial Grams X X^H of X (m x n, ld m, m = m_mul * *m_ptr <= mcap
// <= 128) on the tensor cores (split 1: TF32 operands; 3: 3xTF32), in the
// partial format of the CUDA-core Gram pass; returns the number of partials
int tc_gram(const float2* X, const int* m_ptr, int m_mul, int mcap, long long n, int split,
            float2* gram_part, int ldp, int max_parts, int* status, cudaStream_t s);

// ------------------------------------------------------------- full
template <typename T>
qtt_status tt_full(const qtt_tensor* t, T* y, cudaStream_t s);

// ------------------------------------------------------------- permutations
template <typename T>
void launch_morton_gather(const T* img, T* v, int dx, int dy, int interleave, cudaStream_t s);

// ------------------------------------------------------------- operator
qtt_status op_sinc_create(int d, double B, int normalize, double eps_op, qtt_dtype dt,
                          cudaStream_t s, qtt_op** out);
qtt_status op_embed_axis(const qtt_op* op1d, const TensorDesc& desc, int axis, cudaStream_t s,
                         qtt_op** out);
void op_free(qtt_op* op);

// ------------------------------------------------------------- conv / rounding
qtt_status matvec(const qtt_op* op, const qtt_tensor* x, cudaStream_t s, qtt_tensor** out);
// QTT-FFT / QTT-iFFT of x (QTT_C64), every stage rounded by round_product
// with the identity operator id (k_fft.cu)
qtt_status fft_transform(const qtt_tensor* x, int inverse, const qtt_trunc& tr, const qtt_op* id,
                         int sketch, unsigned long long seed, cudaStream_t s, qtt_tensor** out);
// Sec. 2 padded kernel samples of the sinc (k_op.cu)
qtt_status sinc_padded(int log2_n, long long N, double B, int normalize, qtt_dtype dt, void* g,
                       cudaStream_t s);
// entrywise product, ranks multiply (k_fft.cu)
qtt_status hadamard(const qtt_tensor* x, const qtt_tensor* y, cudaStream_t s, qtt_tensor** out);
qtt_status round_product(const qtt_op* op, const qtt_tensor* x, const qtt_trunc& tr, int sketch,
                         unsigned long long seed, cudaStream_t s, qtt_tensor** out);

// environment sweeps (k_env.cu): dot_out (device, may be null) receives
// <f, w> = sum conj(f) w; grad (d device pointers, may be null) receives
// grad_k = alpha * E_{k-1} W_k R_k + beta * grad_k
qtt_status env_sweep(const qtt_tensor* f, const qtt_tensor* w, double alpha, double beta,
                     void* const* grad, double2* dot_out, cudaStream_t s);
// alpha x + beta y (ranks add)
qtt_status tt_add(double alpha, const qtt_tensor* x, double beta, const qtt_tensor* y,
                  cudaStream_t s, qtt_tensor** out);
// operator with j and i swapped in every core (the adjoint of a real operator)
qtt_status op_transpose(const qtt_op* op, cudaStream_t s, qtt_op** out);

// the cached 1D sinc operator plan for (d, B, normalize, eps_op, dt) (api.cu)
qtt_status cached_op_plan(int d, double B, int normalize, double eps_op, qtt_dtype dt,
                          cudaStream_t s, qtt_op** out);

// drop the cached sketch cores of the rounding (k_round.cu)
void sketch_cache_clear();

// write host-known ranks (<= 32 modes) to a device rank array, stream-ordered
void set_ranks_from_host(int* dev_ranks, const std::vector<int>& r, cudaStream_t s);
// stream-ordered release of a handle
void tensor_free_async(qtt_tensor* t, cudaStream_t s);

// optional per-launch CUDA-event timing (qtt_profile_enable)
struct ProfScope {
  ProfScope(const char* name, cudaStream_t s);
  ~ProfScope();
  const char* name_;
  cudaStream_t s_;
  bool active_;
  void* a_ = nullptr;
  void* b_ = nullptr;
};
#define QTT_PROF_CAT2(a, b) a##b
#define QTT_PROF_CAT(a, b) QTT_PROF_CAT2(a, b)
#define QTT_PROF(name, s) ::qtt::ProfScope QTT_PROF_CAT(_qtt_prof_, __LINE__)(name, s)
// algorithmic flops / bytes of one launch, summed per kernel name while
// profiling is on (qtt_profile_work)
void prof_add_work(const char* name, double flops, double bytes);

// stream-ordered scratch allocation
void* scratch_alloc(size_t bytes, cudaStream_t s);
// record the handle's last-use event on s (no allocation: the event exists
// from tensor_alloc on)
void tensor_stamp(const qtt_tensor* t, cudaStream_t s);
void scratch_free(void* p, cudaStream_t s);

}  // namespace qtt
