// Autotuner for the padded lengths of the free axes and the tile width of the
// generic passes.
//
// Any padded length L >= 2n - 1 of a free axis gives the same physical result
// (§2), but the cost of the transforms depends on L: a power of two selects
// the register-resident kernels, other smooth lengths use fewer or cheaper
// radix stages than 2n when 2n has a large prime factor. The tuner times one
// plan per candidate on the device and keeps the fastest; then, if the plan
// runs any pass on the generic kernels, it times narrower generic tiles (at
// most 8 and 4 lines instead of 16 for FP32, 4 and 2 instead of 8 for FP64:
// more CTAs per line set, shorter per-CTA chains) at those lengths. Results
// are kept in memory, and in a text file when PS_TUNE_CACHE names one (one
// line per geometry: "n1 n2 n3 bc1 bc2 bc3 dtype sms L1 L2 L3 tile", tile 0
// for the default).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace ps {
namespace {

std::mutex g_tune_mu;
std::map<std::string, std::vector<int>> g_tuned;
bool g_file_loaded = false;

bool smooth(int v, const int* primes, int np) {
  for (int i = 0; i < np; ++i)
    while (v % primes[i] == 0) v /= primes[i];
  return v == 1;
}

int next_smooth(int lo, const int* primes, int np) {
  for (int v = lo; v <= kMaxLen; ++v)
    if (smooth(v, primes, np)) return v;
  return 0;
}

void load_file() {
  if (g_file_loaded) return;
  g_file_loaded = true;
  const char* path = getenv("PS_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  int n[3], bc[3], dt, sms, L[3], tile;
  while (fscanf(f, "%d %d %d %d %d %d %d %d %d %d %d %d", &n[0], &n[1], &n[2], &bc[0], &bc[1], &bc[2], &dt, &sms,
                &L[0], &L[1], &L[2], &tile) == 12) {
    char key[128];
    snprintf(key, sizeof key, "%d %d %d %d %d %d %d %d", n[0], n[1], n[2], bc[0], bc[1], bc[2], dt, sms);
    g_tuned[key] = {L[0], L[1], L[2], tile};
  }
  fclose(f);
}

void append_file(const std::string& key, const int* L) {
  const char* path = getenv("PS_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %d\n", key.c_str(), L[0], L[1], L[2], L[3]);
  fclose(f);
}

}  // namespace
}  // namespace ps

extern "C" int ps_plan_autotune(ps_plan p, int reps, void* stream) {
  using namespace ps;
  if (!p) {
    set_error("plan is NULL");
    return PS_ERR_ARG;
  }
  if (p->built) {
    set_error("autotune must run before ps_kernel_build");
    return PS_ERR_ARG;
  }
  if (reps < 1) reps = 5;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    set_error("device query: %s", cudaGetErrorString(e));
    return PS_ERR_CUDA;
  }
  char keybuf[128];
  snprintf(keybuf, sizeof keybuf, "%d %d %d %d %d %d %d %d", p->n[0], p->n[1], p->n[2], p->bc[0], p->bc[1],
           p->bc[2], p->dtype, sms);
  const std::string key(keybuf);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_file();
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      p->gen_tk_max = it->second[3];
      return ps_plan_set_lengths(p, it->second[0], it->second[1], it->second[2]);
    }
  }

  // candidate length triples: one rule applied to every free axis
  static const int p2[] = {2}, p23[] = {2, 3}, p2357[] = {2, 3, 5, 7};
  std::vector<std::vector<int>> cands;
  for (int rule = 0; rule < 4; ++rule) {
    std::vector<int> L(3);
    bool ok = true;
    for (int j = 0; j < 3; ++j) {
      if (p->bc[j] == PS_BC_PERIODIC) {
        L[j] = p->n[j];
        continue;
      }
      const int lo = 2 * p->n[j] - 1;
      switch (rule) {
        case 0: L[j] = 2 * p->n[j]; break;
        case 1: L[j] = next_smooth(lo, p2, 1); break;
        case 2: L[j] = next_smooth(lo, p23, 2); break;
        default: L[j] = next_smooth(lo, p2357, 4); break;
      }
      ok &= L[j] > 0 && L[j] <= kMaxLen;
    }
    L.push_back(0);  // default tile width
    if (ok && std::find(cands.begin(), cands.end(), L) == cands.end()) cands.push_back(L);
  }

  const size_t bytes = (size_t)p->n[0] * p->n[1] * p->n[2] * p->esz;
  void *rho = nullptr, *V = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMalloc(&rho, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&V, bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(rho, 0, bytes, s);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float best_ms = -1.f;
  std::vector<int> best = {p->L[0], p->L[1], p->L[2], 0};
  bool best_generic = false;  // the best plan runs a pass on the generic kernels
  int rc = PS_OK;
  const size_t nlen = cands.size();
  for (size_t c = 0; e == cudaSuccess && rc == PS_OK && c < cands.size(); ++c) {
    if (c == nlen && best_generic) {
      // second phase: narrower generic tiles at the best lengths
      const int t0w = p->dtype == PS_F32 ? 16 : 8;
      for (int tw = t0w / 2; tw >= t0w / 4; tw /= 2) cands.push_back({best[0], best[1], best[2], tw});
      if (c == cands.size()) break;
    } else if (c == nlen) {
      break;
    }
    ps_plan trial = nullptr;
    rc = ps_plan_create(p->n[0], p->n[1], p->n[2], p->h, p->bc[0], p->bc[1], p->bc[2], p->dtype, &trial);
    if (rc == PS_OK) rc = ps_plan_set_lengths(trial, cands[c][0], cands[c][1], cands[c][2]);
    if (rc == PS_OK) trial->gen_tk_max = cands[c][3];
    if (rc == PS_OK) rc = ps_kernel_build(trial, stream);
    for (int w = 0; rc == PS_OK && w < 2; ++w) rc = ps_solve(trial, rho, V, nullptr, stream);
    if (rc == PS_OK) {
      e = cudaEventRecord(t0, s);
      for (int r = 0; rc == PS_OK && r < reps; ++r) rc = ps_solve(trial, rho, V, nullptr, stream);
      if (e == cudaSuccess) e = cudaEventRecord(t1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float ms = 0.f;
      if (e == cudaSuccess && rc == PS_OK) e = cudaEventElapsedTime(&ms, t0, t1);
      if (e == cudaSuccess && rc == PS_OK && (best_ms < 0.f || ms < best_ms)) {
        best_ms = ms;
        best = cands[c];
        best_generic = false;
        for (int k = 0; k < 5; ++k) best_generic |= !trial->cfg[k].fast;
      }
    }
    if (trial) ps_plan_destroy(trial);
  }
  if (rho) cudaFree(rho);
  if (V) cudaFree(V);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (rc != PS_OK) return rc;
  if (e != cudaSuccess) {
    set_error("autotune: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA;
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[key] = best;
    append_file(key, best.data());
  }
  p->gen_tk_max = best[3];
  return ps_plan_set_lengths(p, best[0], best[1], best[2]);
}
