// Batched assembly of several crystals of uneven size as one CUDA graph, built on the first
// call for a given list of (context, H) and schedule and replayed afterwards, so the host
// issues a single launch.  The systems are ordered by their estimated work, smallest first.
// Two schedules:
// The systems are dealt in that order to two chains that run concurrently (forked from and
// joined back into the caller's stream), so the second chain fills the SMs a chain's small
// kernels leave idle.  Per chain, two schedules:
//  - work list: the chain's (system, q-slab) units are packed into steps and each step's
//    tensor-core GEMMs of all its systems run as one grouped persistent launch over their
//    tiles (k_split.cu:split_batch_worklist);
//  - chains: each system's own assembly in turn.
// Either way small systems are not queued behind large ones (shortest-job-first order
// minimises the mean completion time).  A device timestamp (%globaltimer) is written when the
// graph starts and when each system's assembly ends, which gives per-system completion times
// inside the batch.
#include <algorithm>
#include <mutex>
#include <numeric>
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
  int schedule = BSE_BATCH_WORKLIST;
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

// The work-list schedule's launches for the systems ctxs[sub[..]] on `st` (each context
// temporarily bound to it).
bse_status enqueue_worklist(BatchGraph *b, bse_ctx **ctxs, void **H, const std::vector<int> &sub, cudaStream_t st,
                            bool stamps) {
  const int m = (int)sub.size();
  std::vector<cudaStream_t> saved(m);
  std::vector<bool> prof(m);
  for (int r = 0; r < m; r++) {
    bse_ctx *c = ctxs[sub[r]];
    saved[r] = c->stream;
    prof[r] = c->prof;
    c->stream = st;
    c->prof = false;
  }
  const bse_status s = split_batch_worklist(ctxs, H, sub.data(), m, [&](int i) {
    if (!stamps) return;
    k_stamp<<<1, 32, 0, st>>>(b->d_stamps + i + 1);
    bse_count_launch();
  });
  for (int r = 0; r < m; r++) {
    ctxs[sub[r]]->stream = saved[r];
    ctxs[sub[r]]->prof = prof[r];
  }
  return s;
}

// One chain's systems (sub, smallest first) on stream br: the work list, or each system's own
// assembly in turn.
bse_status enqueue_chain(BatchGraph *b, bse_ctx **ctxs, void **H, const std::vector<int> &sub, cudaStream_t br,
                         bool stamps) {
  if (sub.empty()) return BSE_OK;
  if (b->schedule == BSE_BATCH_WORKLIST) return enqueue_worklist(b, ctxs, H, sub, br, stamps);
  for (int i : sub) {
    bse_ctx *c = ctxs[i];
    cudaStream_t saved = c->stream;
    const bool prof = c->prof;
    c->stream = br;
    c->prof = false;
    const bse_status s = bse_assemble(c, H[i]);
    if (stamps) {
      k_stamp<<<1, 32, 0, br>>>(b->d_stamps + i + 1);
      bse_count_launch();
    }
    c->stream = saved;
    c->prof = prof;
    if (s != BSE_OK) return s;
  }
  return BSE_OK;
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
  // estimated work of each assembly: the direct term's M_vv W(q) GEMM and second contraction
  // over all pairs, the exchange over the full square (flops up to a common factor)
  std::vector<double> work(n);
  for (int i = 0; i < n; i++) {
    const bse_ctx *c = ctxs[i];
    const double nk = c->nk, na = c->naux_tot, nv = c->nv, nc = c->nc, dim = (double)c->dim;
    work[i] = nk * nk * nv * nv * (na * na + nc * nc * na) + dim * dim * na;
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b2) { return work[a] < work[b2]; });
  // systems dealt in order to two chains
  const int n_chains = std::min(n, 2);
  std::vector<std::vector<int>> chain(n_chains);
  for (int r = 0; r < n; r++) chain[r % n_chains].push_back(order[r]);
  if (b->schedule == BSE_BATCH_WORKLIST) {
    // eager pass of the grouped launches (sets their attributes outside the capture)
    for (const auto &sub : chain) {
      const bse_status s = enqueue_worklist(b, ctxs, H, sub, stream, false);
      if (s != BSE_OK) return s;
    }
    if (cudaStreamSynchronize(stream) != cudaSuccess) return bse_fail(c0, BSE_ECUDA, "batch: warm-up failed");
  }
  b->branches.resize(n_chains);
  b->events.resize(n_chains + 1);
  for (int i = 0; i < n_chains; i++) cudaStreamCreateWithFlags(&b->branches[i], cudaStreamNonBlocking);
  for (int i = 0; i <= n_chains; i++) cudaEventCreateWithFlags(&b->events[i], cudaEventDisableTiming);
  const long long launches0 = bse_launch_count();
  {
    const cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
      return bse_fail(c0, BSE_ECUDA, std::string("batch: cannot begin stream capture: ") + cudaGetErrorString(e));
  }
  bse_status s = BSE_OK;
  k_stamp<<<1, 32, 0, stream>>>(b->d_stamps);
  bse_count_launch();
  cudaEventRecord(b->events[n_chains], stream);
  for (int ch = 0; ch < n_chains; ch++) cudaStreamWaitEvent(b->branches[ch], b->events[n_chains], 0);
  for (int ch = 0; ch < n_chains && s == BSE_OK; ch++) s = enqueue_chain(b, ctxs, H, chain[ch], b->branches[ch], true);
  for (int ch = 0; ch < n_chains; ch++) {
    cudaEventRecord(b->events[ch], b->branches[ch]);
    cudaStreamWaitEvent(stream, b->events[ch], 0);
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

bse_status bse_batch_assemble(bse_ctx **ctxs, void **H, int n, void *cuda_stream, int32_t schedule,
                              int64_t *stamps_ns) {
  if (!ctxs || !H || n < 1) return BSE_EINVAL;
  if (schedule != BSE_BATCH_WORKLIST && schedule != BSE_BATCH_CHAINS) return BSE_EINVAL;
  for (int i = 0; i < n; i++) {
    if (!ctxs[i] || !H[i]) return BSE_EINVAL;
    if (ctxs[i]->stage < 2) return bse_fail(ctxs[i], BSE_ESTATE, "batch: assemble before project_pairs");
    if (ctxs[i]->device != ctxs[0]->device) return bse_fail(ctxs[i], BSE_EINVAL, "batch: contexts on different devices");
    if (schedule == BSE_BATCH_WORKLIST &&
        (ctxs[i]->precision == BSE_FP64 || ctxs[i]->precision != ctxs[0]->precision))
      return bse_fail(ctxs[i], BSE_EINVAL, "batch: the work-list schedule needs one split precision for all systems");
  }
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  BatchGraph *b = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (BatchGraph *g : g_batches) {
      if (g->stream != stream || g->schedule != schedule || (int)g->ctxs.size() != n) continue;
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
      b->schedule = schedule;
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

bse_status bse_autotune(bse_ctx *c, int *chosen_tile, int *chosen_proj_threads) {
  if (!c) return BSE_EINVAL;
  if (c->precision == BSE_FP64) {
    if (chosen_tile) *chosen_tile = 0;
    if (chosen_proj_threads) *chosen_proj_threads = 0;
    return BSE_OK;
  }
  if (c->stage < 2) return bse_fail(c, BSE_ESTATE, "autotune before project_pairs");
  return split_autotune(c, chosen_tile, chosen_proj_threads);
}

}  // extern "C"
