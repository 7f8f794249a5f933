// Batched TEBD layers: all bonds of one parity of several resident states at once.
//
// The bonds of one layer are independent (Fig. 2a), within a state and across
// states. The executor spreads them over a pool of library-owned worker streams,
// each with its own bond-update workspace, so that the latency-bound parts of
// different updates (the cluster QR panels use up to 16 SMs each) run side by side
// on different SMs while tensor-core contractions fill the rest. The states'
// streams are joined to the workers through events before and after the layer.
//
// For the plain scheme a layer does not synchronise with the host, so a layer whose
// shapes repeat (the saturated-chi regime) is captured into a CUDA graph the second
// time it is seen and replayed afterwards, removing the per-kernel launch cost.
// CBE reads the new bond dimension back after each update and is not captured.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "mps_impl.cuh"

namespace qrtebd {
namespace {

constexpr int kWorkers = 16;
// Bonds whose workspace exceeds QRTEBD_LAYER_BIG_BOND_BYTES run on the first
// QRTEBD_LAYER_BIG_WORKERS workers only, so the executor holds at most that many of the largest
// workspaces (a chi = 1024, d = 5 bond needs ~3 GB); the other bonds of such a layer take the
// remaining workers.
constexpr size_t kBigBond = QRTEBD_LAYER_BIG_BOND_BYTES;
constexpr int kBigWorkers = QRTEBD_LAYER_BIG_WORKERS;
static_assert(kBigWorkers >= 1 && kBigWorkers < kWorkers, "big-bond workers");

struct Worker {
  cudaStream_t st = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cudaEvent_t done = nullptr;
};

struct GraphEntry {
  std::vector<long long> key;
  cudaGraphExec_t exec = nullptr;
  int seen = 0;
  int nkernels = 0;  // kernel nodes, for the launch counter
};

struct Executor {
  int device = -1;
  Worker w[kWorkers];
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  std::vector<cudaEvent_t> state_ev;
  std::vector<GraphEntry> graphs;
  std::mutex mu;
};

Executor g_exec[64];

int executor_init(Executor& ex, int dev) {
  if (ex.device == dev) return QRTEBD_OK;
  for (auto& w : ex.w) {
    QR_CUDA_TRY(cudaStreamCreateWithFlags(&w.st, cudaStreamNonBlocking));
    QR_CUDA_TRY(cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming));
  }
  QR_CUDA_TRY(cudaStreamCreateWithFlags(&ex.origin, cudaStreamNonBlocking));
  QR_CUDA_TRY(cudaEventCreateWithFlags(&ex.fork, cudaEventDisableTiming));
  QR_CUDA_TRY(cudaEventCreateWithFlags(&ex.join, cudaEventDisableTiming));
  ex.device = dev;
  return QRTEBD_OK;
}

void drop_graphs(Executor& ex) {
  for (auto& g : ex.graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  ex.graphs.clear();
}

// A replayed graph holds raw device pointers: any reallocation invalidates them.
int worker_reserve(Executor& ex, Worker& w, size_t need) {
  if (need <= w.ws_bytes) return QRTEBD_OK;
  drop_graphs(ex);
  QR_CUDA_TRY(cudaStreamSynchronize(w.st));
  if (w.ws) cudaFree(w.ws);
  w.ws = nullptr;
  w.ws_bytes = 0;
  if (cudaMalloc(&w.ws, need) != cudaSuccess) {
    (void)cudaGetLastError();
    set_last_message("batched layer: workspace allocation failed");
    return QRTEBD_ERR_OOM;
  }
  w.ws_bytes = need;
  return QRTEBD_OK;
}

struct Task { qrtebd_mps* s; int m; int worker; };

// Enqueue every update of the layer on the workers (fork from `origin`, join back).
int enqueue_layer(Executor& ex, std::vector<Task>& tasks, const qrtebd_trunc* tr) {
  ConcurrencyScope conc((int)std::min<size_t>(tasks.size(), kWorkers));
  QR_CUDA_TRY(cudaEventRecord(ex.fork, ex.origin));
  for (auto& w : ex.w) QR_CUDA_TRY(cudaStreamWaitEvent(w.st, ex.fork, 0));
  for (auto& t : tasks) {
    Worker& w = ex.w[t.worker];
    QR_TRY(mps_update_bond(t.s, t.m, tr, w.st, w.ws, w.ws_bytes));
  }
  for (auto& w : ex.w) {
    QR_CUDA_TRY(cudaEventRecord(w.done, w.st));
    QR_CUDA_TRY(cudaStreamWaitEvent(ex.origin, w.done, 0));
  }
  return QRTEBD_OK;
}

}  // namespace

// Called when a state is destroyed: graphs that captured its buffers must never replay.
void executor_forget_state(qrtebd_mps* s) {
  for (auto& ex : g_exec) {
    if (ex.device < 0) continue;
    std::lock_guard<std::mutex> lk(ex.mu);
    const long long tag = reinterpret_cast<long long>(s);
    std::vector<GraphEntry> keep;
    for (auto& g : ex.graphs) {
      if (std::find(g.key.begin(), g.key.end(), tag) != g.key.end()) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
      } else {
        keep.push_back(g);
      }
    }
    ex.graphs.swap(keep);
  }
}

}  // namespace qrtebd

using namespace qrtebd;

extern "C" {

int qrtebd_layer_workers(void) { return kWorkers; }

int qrtebd_apply_gate_layer_batched(qrtebd_mps* const* states, int nstates, int parity,
                                    const double* const* gates_host, const qrtebd_trunc* tr,
                                    double* const* eps_out) {
  if (!states || nstates < 1 || !gates_host || !tr || (parity != 0 && parity != 1))
    return QRTEBD_ERR_INVALID_ARG;
  for (int i = 0; i < nstates; ++i) {
    if (!states[i] || !gates_host[i]) return QRTEBD_ERR_INVALID_ARG;
    for (int k = 0; k < i; ++k)
      if (states[k] == states[i]) return QRTEBD_ERR_INVALID_ARG;  // a state appears once
  }
  int dev = 0;
  QR_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return QRTEBD_ERR_INVALID_ARG;
  Executor& ex = g_exec[dev];
  std::lock_guard<std::mutex> lk(ex.mu);
  QR_TRY(executor_init(ex, dev));

  // tasks, round-robin over the workers (the largest bonds over the first kBigWorkers only),
  // and the workspace each worker needs
  std::vector<Task> tasks;
  std::vector<size_t> task_need;
  size_t need[kWorkers] = {};
  auto bits = [](double v) { long long b; std::memcpy(&b, &v, sizeof b); return b; };
  std::vector<long long> key = {parity, tr->scheme, tr->chi_max, tr->eta, tr->dchi_min,
                                tr->eps_explicit, tr->reorth, tr->sweeps, bits(tr->dchi_frac),
                                bits(tr->svd_min), bits(tr->tie_tol), bits(tr->eps_target)};
  bool any_big = false;
  for (int i = 0; i < nstates; ++i) {
    qrtebd_mps* s = states[i];
    key.push_back(reinterpret_cast<long long>(s));
    for (int b : s->chi) key.push_back(b);
    for (char c : s->xi_diag) key.push_back(c);
    for (char c : s->xi_lower) key.push_back(c);
    for (int m = parity; m < mps_gate_count(s); m += 2) {
      size_t nb = 0;
      QR_TRY(mps_bond_ws_need(s, m, tr, &nb));
      any_big = any_big || nb > kBigBond;
      tasks.push_back(Task{s, m, 0});
      task_need.push_back(nb);
    }
  }
  int rr_big = 0, rr_small = 0;
  for (size_t t = 0; t < tasks.size(); ++t) {
    int wk;
    if (task_need[t] > kBigBond) wk = rr_big++ % kBigWorkers;
    else if (any_big) wk = kBigWorkers + rr_small++ % (kWorkers - kBigWorkers);
    else wk = rr_small++ % kWorkers;
    tasks[t].worker = wk;
    need[wk] = std::max(need[wk], task_need[t]);
  }
  for (int k = 0; k < kWorkers; ++k) QR_TRY(worker_reserve(ex, ex.w[k], need[k]));

  // gates, then order the origin after every state's earlier work
  if ((int)ex.state_ev.size() < nstates) {
    size_t old = ex.state_ev.size();
    ex.state_ev.resize(nstates);
    for (size_t i = old; i < ex.state_ev.size(); ++i)
      QR_CUDA_TRY(cudaEventCreateWithFlags(&ex.state_ev[i], cudaEventDisableTiming));
  }
  for (int i = 0; i < nstates; ++i) {
    QR_TRY(mps_upload_gates(states[i], parity, gates_host[i]));
    QR_CUDA_TRY(cudaEventRecord(ex.state_ev[i], states[i]->st));
    QR_CUDA_TRY(cudaStreamWaitEvent(ex.origin, ex.state_ev[i], 0));
  }

  // a CBE layer keeps its cuts on the device (collected after the join), so it can be recorded
  // too; in complex128 only while every eta the states can reach fits the one-sided FP64
  // solver (the two-sided fallback synchronises with the host once per sweep)
  bool capturable = (tr->scheme == QRTEBD_PLAIN);
  if (tr->scheme == QRTEBD_CBE) {
    capturable = true;
    for (int i = 0; i < nstates; ++i) {
      const qrtebd_mps* s = states[i];
      if (!prec_is_c128(s->precision)) continue;
      long long dchi = (long long)std::ceil(tr->dchi_frac * s->chi_max - 1e-9);
      if (dchi < tr->dchi_min) dchi = tr->dchi_min;
      const long long eta_cap = std::min<long long>((long long)s->d * s->chi_max, s->chi_max + dchi);
      capturable = capturable && eta_cap <= (1 << 20) && svd64_supported((int)eta_cap);
    }
  }
  GraphEntry* ge = nullptr;
  if (capturable) {
    for (auto& g : ex.graphs)
      if (g.key == key) ge = &g;
    if (!ge) {
      if (ex.graphs.size() >= 16) {
        if (ex.graphs.front().exec) cudaGraphExecDestroy(ex.graphs.front().exec);
        ex.graphs.erase(ex.graphs.begin());
      }
      ex.graphs.push_back(GraphEntry{key, nullptr, 0});
      ge = &ex.graphs.back();
    }
    ge->seen++;
  }
  if (ge && ge->exec) {
    QR_CUDA_TRY(cudaGraphLaunch(ge->exec, ex.origin));
    note_launch(ge->nkernels);
    // host bookkeeping the graph does not do: new bond dimensions (plain: eta; CBE: the cut
    // on the device, collected after the join)
    for (auto& t : tasks) {
      qrtebd_mps* s = t.s;
      const int bl = s->infinite ? t.m % s->L : t.m;
      const int bmid = s->infinite ? (t.m + 1) % s->L : t.m + 1;
      const int br = s->infinite ? (t.m + 2) % s->L : t.m + 2;
      if (tr->scheme == QRTEBD_CBE) {
        s->chi_pending[bmid] = 1;
        s->xi_lower[bmid] = 0;
        continue;
      }
      qrtebd_trunc tt = *tr;
      if (tt.chi_max > s->cap[bmid]) tt.chi_max = s->cap[bmid];
      s->chi[bmid] = choose_eta(&tt, s->chi[bl], s->d, s->chi[bmid], s->chi[br]);
      s->xi_diag[bmid] = 0;
      s->xi_lower[bmid] = 1;
    }
  } else if (ge && ge->seen >= 2) {
    // second sighting of this shape: capture, then launch
    ProfSuppress no_events;
    // the host bookkeeping of the enqueue (bond dimensions) is kept so that a capture that
    // fails can be undone and the layer run without a graph
    std::vector<std::vector<int>> chi_before(nstates);
    std::vector<std::vector<char>> diag_before(nstates), lower_before(nstates), pend_before(nstates);
    for (int i = 0; i < nstates; ++i) {
      chi_before[i] = states[i]->chi;
      diag_before[i] = states[i]->xi_diag;
      lower_before[i] = states[i]->xi_lower;
      pend_before[i] = states[i]->chi_pending;
    }
    QR_CUDA_TRY(cudaStreamBeginCapture(ex.origin, cudaStreamCaptureModeRelaxed));
    int rc = enqueue_layer(ex, tasks, tr);
    cudaGraph_t graph = nullptr;
    cudaError_t ec = cudaStreamEndCapture(ex.origin, &graph);
    if (rc != QRTEBD_OK || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      // worker streams drawn into the failed capture leave it too
      for (auto& w : ex.w) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(w.st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
          cudaGraph_t g2 = nullptr;
          if (cudaStreamEndCapture(w.st, &g2) == cudaSuccess && g2) cudaGraphDestroy(g2);
        }
      }
      (void)cudaGetLastError();
      if (rc != QRTEBD_OK && ec == cudaSuccess) return rc;  // a real failure of the enqueue
      for (int i = 0; i < nstates; ++i) {
        states[i]->chi = chi_before[i];
        states[i]->xi_diag = diag_before[i];
        states[i]->xi_lower = lower_before[i];
        states[i]->chi_pending = pend_before[i];
      }
      ge->seen = -(1 << 30);  // never capture this shape again
      QR_TRY(enqueue_layer(ex, tasks, tr));
      graph = nullptr;
    }
    if (!graph) {
      // ran without a graph (capture refused)
    } else {
    // the capture already updated the host bond dimensions; the graph has not run yet
    size_t nn = 0;
    QR_CUDA_TRY(cudaGraphGetNodes(graph, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) QR_CUDA_TRY(cudaGraphGetNodes(graph, nodes.data(), &nn));
    ge->nkernels = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++ge->nkernels;
    }
    QR_CUDA_TRY(cudaGraphInstantiate(&ge->exec, graph, 0));
    cudaGraphDestroy(graph);
    QR_CUDA_TRY(cudaGraphLaunch(ge->exec, ex.origin));
    }
  } else {
    QR_TRY(enqueue_layer(ex, tasks, tr));
  }

  QR_CUDA_TRY(cudaEventRecord(ex.join, ex.origin));
  for (int i = 0; i < nstates; ++i) QR_CUDA_TRY(cudaStreamWaitEvent(states[i]->st, ex.join, 0));
  // CBE: every state's cuts in one read-back per state, after the whole layer
  for (int i = 0; i < nstates; ++i) QR_TRY(mps_collect_cuts(states[i]));

  if (eps_out) {
    for (int i = 0; i < nstates; ++i) {
      if (!eps_out[i]) continue;
      qrtebd_mps* s = states[i];
      const int ng = mps_gate_count(s);
      std::vector<double> le(ng + 1);
      QR_CUDA_TRY(cudaMemcpyAsync(le.data(), s->layer_eps, ng * sizeof(double), cudaMemcpyDeviceToHost, s->st));
      QR_CUDA_TRY(cudaStreamSynchronize(s->st));
      for (int m = parity; m < ng; m += 2) eps_out[i][m] = le[m];
    }
  }
  return QRTEBD_OK;
}

int qrtebd_mps_set_site(qrtebd_mps* s, int site, const double* B_host, int chi_l, int chi_r) {
  if (!s || !B_host || site < 0 || site >= s->L) return QRTEBD_ERR_INVALID_ARG;
  const int bl = site, br = s->infinite ? (site + 1) % s->L : site + 1;
  if (chi_l < 1 || chi_r < 1 || chi_l > s->cap[bl] || chi_r > s->cap[br]) return QRTEBD_ERR_INVALID_ARG;
  const size_t n = (size_t)chi_l * s->d * chi_r;
  if (prec_is_c128(s->precision)) {
    QR_CUDA_TRY(cudaMemcpyAsync(s->B[site], B_host, n * sizeof(double2), cudaMemcpyHostToDevice, s->st));
  } else {
    std::vector<float2> h(n);
    for (size_t i = 0; i < n; ++i) h[i] = make_float2((float)B_host[2 * i], (float)B_host[2 * i + 1]);
    QR_CUDA_TRY(cudaMemcpyAsync(s->B[site], h.data(), n * sizeof(float2), cudaMemcpyHostToDevice, s->st));
  }
  QR_CUDA_TRY(cudaStreamSynchronize(s->st));
  s->chi[bl] = chi_l;
  s->chi[br] = chi_r;
  return QRTEBD_OK;
}

int qrtebd_mps_set_bond(qrtebd_mps* s, int bond, const double* xi_host, int chi, int diagonal) {
  if (!s || !xi_host || bond < 0 || bond >= s->nbonds_store) return QRTEBD_ERR_INVALID_ARG;
  if (chi < 1 || chi > s->cap[bond]) return QRTEBD_ERR_INVALID_ARG;
  const size_t n = (size_t)chi * chi;
  std::vector<double> dense(2 * n, 0.0);
  if (diagonal) {
    for (int i = 0; i < chi; ++i) { dense[2 * ((size_t)i * chi + i)] = xi_host[2 * i]; dense[2 * ((size_t)i * chi + i) + 1] = xi_host[2 * i + 1]; }
  } else {
    std::memcpy(dense.data(), xi_host, 2 * n * sizeof(double));
  }
  auto put = [&](void* dst, const double* src, size_t cnt) -> int {
    if (prec_is_c128(s->precision)) {
      QR_CUDA_TRY(cudaMemcpyAsync(dst, src, cnt * sizeof(double2), cudaMemcpyHostToDevice, s->st));
    } else {
      std::vector<float2> h(cnt);
      for (size_t i = 0; i < cnt; ++i) h[i] = make_float2((float)src[2 * i], (float)src[2 * i + 1]);
      QR_CUDA_TRY(cudaMemcpyAsync(dst, h.data(), cnt * sizeof(float2), cudaMemcpyHostToDevice, s->st));
      QR_CUDA_TRY(cudaStreamSynchronize(s->st));
    }
    return QRTEBD_OK;
  };
  QR_TRY(put(s->Xi[bond], dense.data(), n));
  if (diagonal) QR_TRY(put(s->xiv[bond], xi_host, chi));
  QR_CUDA_TRY(cudaStreamSynchronize(s->st));
  s->chi[bond] = chi;
  s->xi_diag[bond] = diagonal ? 1 : 0;
  s->xi_lower[bond] = 0;
  return QRTEBD_OK;
}

}  // extern "C"
