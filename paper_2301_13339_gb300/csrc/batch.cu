// Batched lines: many independent 1D signals of uneven length, bandwidth and
// rank cap through decompose -> sinc convolution -> Full in one submission.
//
// Each line's chain is sequential (d small eigen-solves that each occupy one
// SM), so a single line leaves most of the GPU idle.  The batch spreads the
// lines over S internal streams (longest-first onto the least-loaded
// stream), forked from and joined back to the caller's stream with events,
// so up to S chains run at once.  The whole fork/join body can be captured
// once into a CUDA graph and replayed with one launch per batch: the chains
// never wait for the host (ranks stay on the device) and their allocations
// are stream-ordered, so the capture holds every kernel, copy, allocation
// and free of every line.
#include "qtt_internal.cuh"
#include <algorithm>
#include <numeric>
#include <vector>

struct qtt_batch {
  int n = 0;
  std::vector<int> d;
  std::vector<double> B;
  std::vector<int> rmax;
  double eps = 0.0;
  int refine = 1;
  int normalize = 1;
  double eps_op = 1e-7;
  qtt_trunc round_tr{};
  qtt_dtype dt = QTT_C64;
  int nstreams = 0;
  int gram_parts = 0;   // tile settings of the lines' Gram passes (0: defaults)
  int chunk_div = 0;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  std::vector<std::vector<int>> lines_of;   // stream -> lines in submission order
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace qtt {

static qtt_status run_line(qtt_batch* b, int i, const void* x, void* y, cudaStream_t s) {
  qtt_trunc tr{b->eps, b->rmax[i], b->refine, 0.0};
  const int lg = b->d[i];
  qtt_tensor* f = nullptr;
  qtt_status st = qtt_decompose(x, b->dt, 1, &lg, 1, &tr, s, &f);
  if (st != QTT_OK) return st;
  qtt_tensor* yq = nullptr;
  const double Bi = b->B[i];
  st = qtt_conv_sinc(f, &Bi, b->normalize, b->eps_op, &b->round_tr, 0,
                     20230131ULL + (unsigned long long)i, s, &yq);
  tensor_free_async(f, s);
  if (st != QTT_OK) return st;
  st = qtt_to_full(yq, y, s);
  tensor_free_async(yq, s);
  return st;
}

static qtt_status run_all_body(qtt_batch* b, const void* const* x, void* const* y, cudaStream_t s);

// the batch's tile settings hold while its lines are submitted (a captured
// graph keeps the launch shapes it was captured with)
static qtt_status run_all(qtt_batch* b, const void* const* x, void* const* y, cudaStream_t s) {
  set_gram_tiles(b->gram_parts, b->chunk_div);
  const qtt_status st = run_all_body(b, x, y, s);
  set_gram_tiles(0, 0);
  return st;
}

static qtt_status run_all_body(qtt_batch* b, const void* const* x, void* const* y, cudaStream_t s) {
  qtt_status st = cuda_check(cudaEventRecord(b->fork, s), "batch fork");
  if (st != QTT_OK) return st;
  for (int j = 0; j < b->nstreams; ++j) {
    st = cuda_check(cudaStreamWaitEvent(b->streams[j], b->fork, 0), "batch fork wait");
    if (st != QTT_OK) return st;
  }
  for (int j = 0; j < b->nstreams; ++j)
    for (int i : b->lines_of[j]) {
      st = run_line(b, i, x[i], y[i], b->streams[j]);
      if (st != QTT_OK) return st;
    }
  for (int j = 0; j < b->nstreams; ++j) {
    st = cuda_check(cudaEventRecord(b->join[j], b->streams[j]), "batch join");
    if (st != QTT_OK) return st;
    st = cuda_check(cudaStreamWaitEvent(s, b->join[j], 0), "batch join wait");
    if (st != QTT_OK) return st;
  }
  return QTT_OK;
}

static void batch_destroy(qtt_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto s : b->streams) cudaStreamDestroy(s);
  delete b;
}

}  // namespace qtt

using namespace qtt;

extern "C" {

qtt_status qtt_batch_create(int nlines, const int* log2_len, const double* B, const int* rmax,
                            double eps, int refine, int normalize, double eps_op,
                            const qtt_trunc* round_tr, qtt_dtype dt, int nstreams, void* stream,
                            qtt_batch** out) {
  if (!log2_len || !B || !rmax || !round_tr || !out || nlines < 1) {
    set_error("qtt_batch_create: bad argument");
    return QTT_EINVAL;
  }
  if (round_tr->fixed_ranks) {
    set_error("qtt_batch_create: fixed_ranks are not supported for batches (lines differ in length)");
    return QTT_EINVAL;
  }
  if (round_tr->prec == QTT_PREC_BF16_REFINED || round_tr->prec == QTT_PREC_TF32_REFINED) {
    set_error("qtt_batch_create: the BF16/TF32 tensor-core precision modes are not built");
    return QTT_EUNSUPPORTED;
  }
  if (dt == QTT_F32 || dt == QTT_C128) {
    set_error("qtt_batch_create: element type %d is not built (QTT_F64 and QTT_C64 are)", (int)dt);
    return QTT_EUNSUPPORTED;
  }
  if (dt != QTT_C64 && dt != QTT_F64) { set_error("qtt_batch_create: dtype"); return QTT_EINVAL; }
  if (!(eps >= 0.0) || eps >= 1.0 || !(eps_op > 0.0) || eps_op >= 1.0) {
    set_error("qtt_batch_create: eps in [0, 1) and eps_op in (0, 1) required");
    return QTT_EINVAL;
  }
  if (nstreams < 1) nstreams = 16;
  nstreams = std::min(nstreams, std::min(nlines, 128));
  for (int i = 0; i < nlines; ++i) {
    if (log2_len[i] < 2 || log2_len[i] > 30 || !(B[i] > 0.0)) {
      set_error("qtt_batch_create: line %d: log2 length in [2, 30] and B > 0 required", i);
      return QTT_EINVAL;
    }
  }
  qtt_batch* b = new qtt_batch();
  b->n = nlines;
  b->d.assign(log2_len, log2_len + nlines);
  b->B.assign(B, B + nlines);
  b->rmax.assign(rmax, rmax + nlines);
  b->eps = eps;
  b->refine = refine ? 1 : 0;
  b->normalize = normalize ? 1 : 0;
  b->eps_op = eps_op;
  b->round_tr = *round_tr;
  b->dt = dt;
  b->nstreams = nstreams;
  qtt_status st = QTT_OK;
  for (int j = 0; j < nstreams && st == QTT_OK; ++j) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    st = cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "batch stream");
    if (st == QTT_OK) b->streams.push_back(s);
    if (st == QTT_OK) st = cuda_check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "batch event");
    if (st == QTT_OK) b->join.push_back(e);
  }
  if (st == QTT_OK) st = cuda_check(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "batch event");
  if (st != QTT_OK) { batch_destroy(b); return st; }
  // longest first onto the least-loaded stream; a line's cost ~ d x rank cap
  std::vector<int> order(nlines);
  std::iota(order.begin(), order.end(), 0);
  auto cost = [&](int i) {
    const int r = b->rmax[i] > 0 ? std::min(b->rmax[i], QTT_RANK_CAP) : QTT_RANK_CAP;
    return (double)b->d[i] * (double)r * (double)r;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost(a) > cost(c); });
  std::vector<double> load(nstreams, 0.0);
  b->lines_of.assign(nstreams, {});
  for (int i : order) {
    const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->lines_of[j].push_back(i);
    load[j] += cost(i);
  }
  // operator plans (synchronising, once per distinct (d, B))
  for (int i = 0; i < nlines && st == QTT_OK; ++i) {
    qtt_op* op = nullptr;
    st = cached_op_plan(b->d[i], b->B[i], b->normalize, b->eps_op, dt, (cudaStream_t)stream, &op);
  }
  if (st != QTT_OK) { batch_destroy(b); return st; }
  *out = b;
  return QTT_OK;
}

qtt_status qtt_batch_run(qtt_batch* b, const void* const* x, void* const* y, void* stream) {
  if (!b || !x || !y) { set_error("qtt_batch_run: NULL argument"); return QTT_EINVAL; }
  return run_all(b, x, y, (cudaStream_t)stream);
}

qtt_status qtt_batch_capture(qtt_batch* b, const void* const* x, void* const* y, void* stream) {
  if (!b || !x || !y) { set_error("qtt_batch_capture: NULL argument"); return QTT_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  if (!s) { set_error("qtt_batch_capture: needs a non-default stream"); return QTT_EINVAL; }
  // one eager run: pool growth, kernel attributes and sketch caches settle
  qtt_status st = run_all(b, x, y, s);
  if (st != QTT_OK) return st;
  st = cuda_check(cudaStreamSynchronize(s), "batch warm-up");
  if (st != QTT_OK) return st;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  st = cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed), "batch begin capture");
  if (st != QTT_OK) return st;
  qtt_status body = run_all(b, x, y, s);
  cudaGraph_t g = nullptr;
  st = cuda_check(cudaStreamEndCapture(s, &g), "batch end capture");
  if (body != QTT_OK) { if (g) cudaGraphDestroy(g); return body; }
  if (st != QTT_OK) return st;
  b->graph = g;
  st = cuda_check(cudaGraphInstantiate(&b->exec, g, 0), "batch instantiate");
  return st;
}

qtt_status qtt_batch_set_tiles(qtt_batch* b, int gram_parts_per_sm, int chunk_div) {
  if (!b) { set_error("qtt_batch_set_tiles: NULL batch"); return QTT_EINVAL; }
  if (gram_parts_per_sm < 0 || gram_parts_per_sm > 16 ||
      !(chunk_div == 0 || chunk_div == 1 || chunk_div == 2 || chunk_div == 4)) {
    set_error("qtt_batch_set_tiles: gram_parts_per_sm in [0, 16], chunk_div in {0, 1, 2, 4}");
    return QTT_EINVAL;
  }
  b->gram_parts = gram_parts_per_sm;
  b->chunk_div = chunk_div > 1 ? chunk_div : 0;
  // a captured graph holds the old shapes: it is dropped (capture again)
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  return QTT_OK;
}

qtt_status qtt_batch_launch(qtt_batch* b, void* stream) {
  if (!b || !b->exec) { set_error("qtt_batch_launch: no captured graph"); return QTT_EINVAL; }
  return cuda_check(cudaGraphLaunch(b->exec, (cudaStream_t)stream), "batch launch");
}

qtt_status qtt_batch_info(const qtt_batch* b, int* nstreams, int* graph_nodes) {
  if (!b) { set_error("qtt_batch_info: NULL"); return QTT_EINVAL; }
  if (nstreams) *nstreams = b->nstreams;
  if (graph_nodes) {
    size_t nn = 0;
    if (b->graph) cudaGraphGetNodes(b->graph, nullptr, &nn);
    *graph_nodes = (int)nn;
  }
  return QTT_OK;
}

void qtt_batch_free(qtt_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  batch_destroy(b);
}

qtt_status qtt_batch_conv_sinc(int nlines, const void* const* x, const int* log2_len,
                               const double* B, const int* rmax, double eps, int refine,
                               int normalize, double eps_op, const qtt_trunc* round_tr,
                               void* const* y, qtt_dtype dt, void* stream) {
  qtt_batch* b = nullptr;
  qtt_status st = qtt_batch_create(nlines, log2_len, B, rmax, eps, refine, normalize, eps_op,
                                   round_tr, dt, 0, stream, &b);
  if (st != QTT_OK) return st;
  st = run_all(b, x, y, (cudaStream_t)stream);
  // the streams are released once their work completes
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto e : b->join) cudaEventDestroy(e);
  cudaEventDestroy(b->fork);
  for (auto s2 : b->streams) cudaStreamDestroy(s2);
  delete b;
  return st;
}

}  // extern "C"
