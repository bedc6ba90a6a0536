// Batched assembly of several crystals of uneven size as one CUDA graph: one branch per
// context, forked from and joined back into the caller's stream, so the GPU interleaves the
// systems' kernels and the host issues a single launch.  The graph is built on the first
// call for a given list of (context, H) and replayed afterwards.  A device timestamp
// (%globaltimer) is written when the graph starts and when each branch ends, which gives
// per-system completion times inside the batch.
#include <mutex>
#include <string>
#include <vector>

#include "bse_internal.cuh"

namespace {

__global__ void k_stamp(unsigned long long *slot) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    *slot = t;
  }
}

struct BatchGraph {
  std::vector<bse_ctx *> ctxs;
  std::vector<void *> H;
  cudaStream_t stream = nullptr;   // the caller's stream (may be the legacy default stream)
  cudaStream_t own = nullptr;      // capture and replay stream, ordered against `stream` by events
  cudaEvent_t in = nullptr, out = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> branches;
  std::vector<cudaEvent_t> events;
  unsigned long long *d_stamps = nullptr;
  long long nodes = 0;  // kernels per replay
};

std::mutex g_batch_mu;
std::vector<BatchGraph *> g_batches;

void destroy(BatchGraph *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->own) cudaStreamDestroy(b->own);
  if (b->in) cudaEventDestroy(b->in);
  if (b->out) cudaEventDestroy(b->out);
  for (auto s : b->branches) cudaStreamDestroy(s);
  for (auto e : b->events) cudaEventDestroy(e);
  if (b->d_stamps) cudaFree(b->d_stamps);
  delete b;
}

bse_status build(BatchGraph *b, bse_ctx **ctxs, void **H, int n, cudaStream_t stream) {
  bse_ctx *c0 = ctxs[0];
  cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking);
  cudaEventCreateWithFlags(&b->in, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&b->out, cudaEventDisableTiming);
  stream = b->own;
  // eager pass: sets every lazily configured kernel attribute outside the capture
  for (int i = 0; i < n; i++) {
    bse_status s = bse_assemble(ctxs[i], H[i]);
    if (s != BSE_OK) return s;
    if (cudaStreamSynchronize(ctxs[i]->stream) != cudaSuccess) return bse_fail(c0, BSE_ECUDA, "batch: warm-up failed");
  }
  if (cudaMalloc((void **)&b->d_stamps, sizeof(unsigned long long) * (n + 1)) != cudaSuccess) {
    cudaGetLastError();
    return bse_fail(c0, BSE_ENOMEM, "batch: timestamp allocation failed");
  }
  b->branches.resize(n);
  b->events.resize(n + 1);
  for (int i = 0; i < n; i++) cudaStreamCreateWithFlags(&b->branches[i], cudaStreamNonBlocking);
  for (int i = 0; i <= n; i++) cudaEventCreateWithFlags(&b->events[i], cudaEventDisableTiming);
  const long long launches0 = bse_launch_count();
  {
    const cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
      return bse_fail(c0, BSE_ECUDA, std::string("batch: cannot begin stream capture: ") + cudaGetErrorString(e));
  }
  bse_status s = BSE_OK;
  k_stamp<<<1, 32, 0, stream>>>(b->d_stamps);
  bse_count_launch();
  cudaEventRecord(b->events[n], stream);
  for (int i = 0; i < n && s == BSE_OK; i++) {
    bse_ctx *c = ctxs[i];
    cudaStreamWaitEvent(b->branches[i], b->events[n], 0);
    cudaStream_t saved = c->stream;
    const bool prof = c->prof;
    c->stream = b->branches[i];
    c->prof = false;
    s = bse_assemble(c, H[i]);
    k_stamp<<<1, 32, 0, b->branches[i]>>>(b->d_stamps + i + 1);
    bse_count_launch();
    c->stream = saved;
    c->prof = prof;
    cudaEventRecord(b->events[i], b->branches[i]);
    cudaStreamWaitEvent(stream, b->events[i], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(stream, &graph);
  b->nodes = bse_launch_count() - launches0;
  bse_count_launch((int)-b->nodes);  // capturing launches nothing; replays count below
  if (s != BSE_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (ec != cudaSuccess || !graph) return bse_fail(c0, BSE_ECUDA, "batch: stream capture failed");
  const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return bse_fail(c0, BSE_ECUDA, "batch: graph instantiation failed");
  return BSE_OK;
}

}  // namespace

extern "C" {

bse_status bse_batch_assemble(bse_ctx **ctxs, void **H, int n, void *cuda_stream, int64_t *stamps_ns) {
  if (!ctxs || !H || n < 1) return BSE_EINVAL;
  for (int i = 0; i < n; i++) {
    if (!ctxs[i] || !H[i]) return BSE_EINVAL;
    if (ctxs[i]->stage < 2) return bse_fail(ctxs[i], BSE_ESTATE, "batch: assemble before project_pairs");
    if (ctxs[i]->device != ctxs[0]->device) return bse_fail(ctxs[i], BSE_EINVAL, "batch: contexts on different devices");
  }
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  BatchGraph *b = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (BatchGraph *g : g_batches) {
      if (g->stream != stream || (int)g->ctxs.size() != n) continue;
      bool same = true;
      for (int i = 0; i < n && same; i++) same = g->ctxs[i] == ctxs[i] && g->H[i] == H[i];
      if (same) {
        b = g;
        break;
      }
    }
    if (!b) {
      b = new BatchGraph();
      b->ctxs.assign(ctxs, ctxs + n);
      b->H.assign(H, H + n);
      b->stream = stream;
      bse_status s = build(b, ctxs, H, n, stream);
      if (s != BSE_OK) {
        destroy(b);
        return s;
      }
      g_batches.push_back(b);
    }
  }
  if (cudaEventRecord(b->in, stream) != cudaSuccess || cudaStreamWaitEvent(b->own, b->in, 0) != cudaSuccess ||
      cudaGraphLaunch(b->exec, b->own) != cudaSuccess || cudaEventRecord(b->out, b->own) != cudaSuccess ||
      cudaStreamWaitEvent(stream, b->out, 0) != cudaSuccess)
    return bse_fail(ctxs[0], BSE_ECUDA, "batch: graph launch failed");
  bse_count_launch((int)b->nodes);
  if (stamps_ns) {
    std::vector<unsigned long long> t(n + 1);
    if (cudaStreamSynchronize(stream) != cudaSuccess ||
        cudaMemcpy(t.data(), b->d_stamps, sizeof(unsigned long long) * (n + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
      return bse_fail(ctxs[0], BSE_ECUDA, "batch: timestamp readback failed");
    for (int i = 0; i < n; i++) stamps_ns[i] = (int64_t)(t[i + 1] - t[0]);
  }
  return BSE_OK;
}

void bse_batch_release(void) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (BatchGraph *g : g_batches) destroy(g);
  g_batches.clear();
}

bse_status bse_autotune(bse_ctx *c, int *chosen_tile) {
  if (!c) return BSE_EINVAL;
  if (c->precision == BSE_FP64) {
    if (chosen_tile) *chosen_tile = 0;
    return BSE_OK;
  }
  return split_autotune(c, chosen_tile);
}

}  // extern "C"
