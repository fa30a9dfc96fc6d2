// Batched solves as one CUDA graph.
//
// The five launches of each problem form a chain; the chains of different
// problems are independent. They are captured once, fanned out over side
// streams so the graph lets different problems' passes run side by side
// (small, uneven problems cannot fill the GPU one at a time), and replayed
// with a single cudaGraphLaunch. Instantiated graphs are cached by the exact
// set of plans and pointers; destroying a plan drops every graph that uses it.
//
// Problems go to the side streams longest first, each to the stream with the
// least estimated work so far (the LPT rule), so that no chain is left
// running alone at the end of the batch (PS_BATCH_ORDER=rr: item i on
// stream i mod 16).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace ps {
namespace {

constexpr int kSideStreams = 16;
constexpr size_t kCacheSize = 8;

struct Entry {
  std::vector<const void*> key;  // device, plans, rho, V, E pointers
  cudaGraphExec_t exec = nullptr;
  unsigned long long last_use = 0;
};

struct Side {
  int device = -1;
  cudaStream_t origin = nullptr;
  cudaStream_t s[kSideStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kSideStreams] = {};
};

std::mutex g_mu;
std::vector<Entry> g_cache;
std::vector<Side> g_side;
unsigned long long g_tick = 0;

cudaError_t side_for(int dev, Side** out) {
  for (Side& sd : g_side)
    if (sd.device == dev) {
      *out = &sd;
      return cudaSuccess;
    }
  Side sd;
  sd.device = dev;
  cudaError_t e = cudaStreamCreateWithFlags(&sd.origin, cudaStreamNonBlocking);
  for (int k = 0; e == cudaSuccess && k < kSideStreams; ++k) e = cudaStreamCreateWithFlags(&sd.s[k], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sd.fork, cudaEventDisableTiming);
  for (int k = 0; e == cudaSuccess && k < kSideStreams; ++k) e = cudaEventCreateWithFlags(&sd.join[k], cudaEventDisableTiming);
  if (e != cudaSuccess) return e;
  g_side.push_back(sd);
  *out = &g_side.back();
  return cudaSuccess;
}

cudaError_t launch_one(ps_plan_s* p, const void* rho, void* V, double* E, cudaStream_t s) {
  if (p->dtype == PS_F32)
    return launch_solve<float>(p, static_cast<const float*>(rho), static_cast<float*>(V), E, s, nullptr);
  return launch_solve<double>(p, static_cast<const double*>(rho), static_cast<double*>(V), E, s, nullptr);
}

// Estimated work of one solve: lines x N log2 N per transform (Bluestein:
// two length-M transforms and the chirp products), forward and inverse.
double solve_cost(const ps_plan_s* p) {
  auto f = [&](int j, int N) -> double {
    if (N < 2) return 0.0;
    const int M = p->blue[j].M;
    return M ? 2.0 * M * std::log2((double)M) + 3.0 * N : N * std::log2((double)N);
  };
  const double n2 = p->n[1], n3 = p->n[2];
  const double x = p->L[0] % 2 == 0 ? n2 * n3 * f(0, p->L[0] / 2) : 0.5 * n2 * n3 * f(0, p->L[0]);
  const double y = (double)p->c * n3 * f(1, p->L[1]);
  const double z = (double)p->c * p->L[1] * f(2, p->L[2]);
  return 2.0 * (x + y + z);
}

cudaError_t capture(int count, ps_plan_s* const* plans, const void* const* rho, void* const* V, double* E,
                    Side* sd, cudaGraphExec_t* exec) {
  const int K = std::min(count, kSideStreams);
  std::vector<int> order(count), stream(count);
  std::iota(order.begin(), order.end(), 0);
  const char* o = getenv("PS_BATCH_ORDER");
  if (o && strcmp(o, "rr") == 0) {
    for (int i = 0; i < count; ++i) stream[i] = i % K;
  } else {
    std::vector<double> cost(count), load(K, 0.0);
    for (int i = 0; i < count; ++i) cost[i] = solve_cost(plans[i]);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    for (int i : order) {
      const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      stream[i] = k;
      load[k] += cost[i];
    }
  }
  cudaError_t e = cudaStreamBeginCapture(sd->origin, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t first = cudaEventRecord(sd->fork, sd->origin);
  for (int k = 0; first == cudaSuccess && k < K; ++k) first = cudaStreamWaitEvent(sd->s[k], sd->fork, 0);
  for (int j = 0; first == cudaSuccess && j < count; ++j) {
    const int i = order[j];
    first = launch_one(plans[i], rho[i], V[i], E ? E + i : nullptr, sd->s[stream[i]]);
  }
  // join every side stream back, even after an error, so the capture can end
  for (int k = 0; k < K; ++k) {
    cudaError_t r = cudaEventRecord(sd->join[k], sd->s[k]);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(sd->origin, sd->join[k], 0);
    if (first == cudaSuccess) first = r;
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(sd->origin, &graph);
  if (first == cudaSuccess) first = e;
  if (first == cudaSuccess) first = cudaGraphInstantiate(exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  return first;
}

}  // namespace

cudaError_t batch_solve_graph(int count, ps_plan_s* const* plans, const void* const* rho, void* const* V,
                              double* E, int device, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_mu);
  std::vector<const void*> key;
  key.reserve(3 * count + 2);
  key.push_back(reinterpret_cast<const void*>(static_cast<uintptr_t>(device)));
  key.push_back(E);
  for (int i = 0; i < count; ++i) {
    key.push_back(plans[i]);
    key.push_back(rho[i]);
    key.push_back(V[i]);
  }
  Entry* hit = nullptr;
  for (Entry& en : g_cache)
    if (en.key == key) hit = &en;
  if (!hit) {
    Side* sd = nullptr;
    cudaError_t e = side_for(device, &sd);
    if (e != cudaSuccess) return e;
    cudaGraphExec_t exec = nullptr;
    e = capture(count, plans, rho, V, E, sd, &exec);
    if (e != cudaSuccess) return e;
    if (g_cache.size() >= kCacheSize) {
      auto lru = std::min_element(g_cache.begin(), g_cache.end(),
                                  [](const Entry& a, const Entry& b) { return a.last_use < b.last_use; });
      cudaGraphExecDestroy(lru->exec);
      g_cache.erase(lru);
    }
    g_cache.push_back(Entry{key, exec, 0});
    hit = &g_cache.back();
  }
  hit->last_use = ++g_tick;
  return cudaGraphLaunch(hit->exec, s);
}

void batch_forget_plan(const ps_plan_s* p) {
  std::lock_guard<std::mutex> lock(g_mu);
  for (size_t i = 0; i < g_cache.size();) {
    const auto& k = g_cache[i].key;
    bool uses = false;
    for (size_t j = 2; j < k.size(); j += 3) uses |= (k[j] == p);
    if (uses) {
      cudaGraphExecDestroy(g_cache[i].exec);
      g_cache.erase(g_cache.begin() + i);
    } else {
      ++i;
    }
  }
}

}  // namespace ps
