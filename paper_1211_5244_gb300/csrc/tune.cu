// Autotuner for the padded lengths of the free axes and the kernel schedule
// of a plan.
//
// Any padded length L >= 2n - 1 of a free axis gives the same physical result
// (§2), but the cost of the transforms depends on L: a power of two or
// 96, 192, 384 select the register-resident kernels, other smooth lengths use fewer or
// cheaper radix stages than 2n when 2n has a large prime factor. The tuner times one
// trial plan per candidate on the device and keeps the fastest, then tunes
// the schedule at those lengths one choice at a time (each kept only if it
// is faster), among the choices that apply to the plan:
//   tile    lines per tile of the generic passes (32 / 16 / 8 / 4 in FP32,
//           16 / 8 / 4 / 2 in FP64: wider tiles give each thread more
//           butterflies per stage, narrower ones more CTAs per line set)
//   radix   radix split of the generic Stockham stages (radix 8 first, or
//           radix 4 and 2 only)
//   tile and radix again per axis: for the generic passes along each
//           physical axis on its own (ps_plan_set_axis_schedule)
//   ztk     lines per tile of the persistent packed z kernel (8 or 16)
//   ykind   y kernels: packed persistent, unpacked persistent, non-persistent
//   xy      the fused x/y passes (thread-block clusters) or the separate ones
//   chunks  the x and y passes whole or in chunks of z planes (L2 reuse)
//   order   the plan's processing order of the axes (§3's rule by default), or
//           x first, which runs the specialised FP32 kernels where the
//           lengths have them (more 1D transforms, faster kernels)
// Results are kept in memory, and in a text file when PS_TUNE_CACHE names one
// (one line per geometry: "n1 n2 n3 bc1 bc2 bc3 mode sms L1 L2 L3 tile radix
// ztk ykind xy xfirst chunks tile_x tile_y tile_z radix_x+1 radix_y+1
// radix_z+1", mode = dtype + 2 math + 4 (the plan's order as 9 a0 + 3 a1 +
// a2), 0 for a default choice).
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

// a tuned choice: padded lengths and the schedule fields of the plan
enum { kL1, kL2, kL3, kTile, kRadix, kZtk, kYkind, kXy, kXfirst, kChunks, kTileAx, kRadixAx = kTileAx + 3,
       kFields = kRadixAx + 3 };

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
  char line[512];
  while (fgets(line, sizeof line, f)) {
    // 8 key fields, then the choice; lines of another field count are skipped
    std::vector<long> w;
    char* q = line;
    while (true) {
      char* end = nullptr;
      const long x = strtol(q, &end, 10);
      if (end == q) break;
      w.push_back(x);
      q = end;
    }
    if (w.size() != (size_t)(8 + kFields)) continue;
    char key[128];
    snprintf(key, sizeof key, "%ld %ld %ld %ld %ld %ld %ld %ld", w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7]);
    g_tuned[key] = std::vector<int>(w.begin() + 8, w.end());
  }
  fclose(f);
}

void append_file(const std::string& key, const std::vector<int>& v) {
  const char* path = getenv("PS_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s", key.c_str());
  for (int x : v) fprintf(f, " %d", x);
  fprintf(f, "\n");
  fclose(f);
}

// applies a tuned choice to an unbuilt plan
int apply_choice(ps_plan p, const std::vector<int>& v) {
  const int rc = ps_plan_set_lengths(p, v[kL1], v[kL2], v[kL3]);
  if (rc != PS_OK) return rc;
  p->gen_tk_max = v[kTile];
  p->radix_pref = v[kRadix];
  p->z_tk = v[kZtk];
  p->y_kind = v[kYkind];
  p->xy_sched = v[kXy];
  p->chunk_req = v[kChunks];
  for (int j = 0; j < 3; ++j) {
    p->tile_ax[j] = v[kTileAx + j];
    p->radix_ax[j] = v[kRadixAx + j] - 1;
  }
  if (v[kXfirst]) return ps_plan_set_order(p, 0, 1, 2);
  return PS_OK;
}

// What a built trial plan says about the choices that apply to it.
struct Applies {
  bool generic = false;  // some pass runs the generic kernels
  bool generic_ax[3] = {false, false, false};  // ... along physical axis j
  bool zpipe = false;    // the z pass runs the persistent packed kernel
  bool ypacked = false;  // the y passes run the packed persistent kernels
  bool xy = false;       // the fused x/y kernels run
  bool chunkable = false;  // the x and y passes may run in chunks of z planes
};

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
           p->bc[2], p->dtype + 2 * p->math + 4 * (9 * p->ord[0] + 3 * p->ord[1] + p->ord[2]), sms);
  const std::string key(keybuf);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_file();
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return apply_choice(p, it->second);
  }

  const size_t bytes = (size_t)p->n[0] * p->n[1] * p->n[2] * p->esz;
  void *rho = nullptr, *V = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMalloc(&rho, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&V, bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(rho, 0, bytes, s);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  int rc = PS_OK;

  // builds a trial plan with choice v and returns in *ms the time per solve:
  // the lesser of two timed runs of at least `reps` solves each, lengthened
  // to about a millisecond for small plans (timing noise would otherwise pick
  // choices at random), after two untimed solves; *ms < 0 if the choice is
  // not valid for this plan
  auto trial = [&](const std::vector<int>& v, float* ms, Applies* ap) {
    *ms = -1.f;
    ps_plan tp = nullptr;
    int r = ps_plan_create(p->n[0], p->n[1], p->n[2], p->h, p->bc[0], p->bc[1], p->bc[2], p->dtype, &tp);
    if (r == PS_OK) r = ps_plan_set_math(tp, p->math);
    if (r == PS_OK) r = ps_plan_set_order(tp, p->ord[0], p->ord[1], p->ord[2]);
    if (r == PS_OK) r = apply_choice(tp, v);
    if (r == PS_OK) r = ps_kernel_build(tp, stream);
    for (int w = 0; r == PS_OK && w < 2; ++w) r = ps_solve(tp, rho, V, nullptr, stream);
    if (r == PS_OK) {
      auto timed = [&](int count, float* out) {
        e = cudaEventRecord(t0, s);
        for (int k = 0; r == PS_OK && k < count; ++k) r = ps_solve(tp, rho, V, nullptr, stream);
        if (e == cudaSuccess) e = cudaEventRecord(t1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess && r == PS_OK) e = cudaEventElapsedTime(out, t0, t1);
        *out /= (float)count;
      };
      float a = 0.f, b = 0.f;
      timed(reps, &a);
      const int count = a > 0.f ? std::min(400, std::max(reps, (int)(1.0f / a) + 1)) : reps;
      if (e == cudaSuccess && r == PS_OK) timed(count, &a);
      if (e == cudaSuccess && r == PS_OK) timed(count, &b);
      *ms = std::min(a, b);
      if (ap) {
        for (int k = 0; k < 5; ++k) {
          ap->generic |= !tp->cfg[k].fast;
          ap->generic_ax[pass_axis(tp, k)] |= !tp->cfg[k].fast;
        }
        ap->zpipe = tp->zsoa_T == 16 && tp->zsoa_P == 16 && tp->cfg[P3].fast && !tp->tctab;
        ap->ypacked = tp->ysoa == 3;
        ap->xy = tp->xyfuse != 0;
        ap->chunkable = !tp->xyfuse && tp->cfg[P1].fast && tp->cfg[P2].fast && tp->cfg[P4].fast &&
                        tp->cfg[P5].fast && tp->cfg[P2].fa.nrows == tp->n[2] && tp->n[2] >= 4;
      }
    }
    if (tp) ps_plan_destroy(tp);
    if (r == PS_ERR_UNSUPPORTED || r == PS_ERR_ARG) r = PS_OK;  // a choice that does not apply
    return r;
  };

  // 1. padded lengths: one rule applied to every free axis (2n; the next
  // power of two; the next 2,3- and 2,3,5,7-smooth lengths; the next length
  // with register kernels, a power of two or 96, 192, 384)
  static const int p2[] = {2}, p23[] = {2, 3}, p2357[] = {2, 3, 5, 7};
  std::vector<std::vector<int>> cands;
  for (int rule = 0; rule < 5; ++rule) {
    std::vector<int> v(kFields, 0);
    bool ok = true;
    for (int j = 0; j < 3; ++j) {
      if (p->bc[j] == PS_BC_PERIODIC) {
        v[j] = p->n[j];
        continue;
      }
      const int lo = 2 * p->n[j] - 1;
      switch (rule) {
        case 0: v[j] = 2 * p->n[j]; break;
        case 1: v[j] = next_smooth(lo, p2, 1); break;
        case 2: v[j] = next_smooth(lo, p23, 2); break;
        case 3: v[j] = next_smooth(lo, p2357, 4); break;
        default: {
          int q = next_smooth(lo, p2, 1);
          for (const int r : {96, 192, 384})
            if (lo <= r && r < q) q = r;
          v[j] = q;
          break;
        }
      }
      ok &= v[j] > 0 && v[j] <= kMaxLen;
    }
    if (ok && std::find(cands.begin(), cands.end(), v) == cands.end()) cands.push_back(v);
  }
  float best_ms = -1.f;
  std::vector<int> best(kFields, 0);
  for (int j = 0; j < 3; ++j) best[kL1 + j] = p->L[j];
  Applies best_ap;
  for (size_t c = 0; e == cudaSuccess && rc == PS_OK && c < cands.size(); ++c) {
    float ms;
    Applies ap;
    rc = trial(cands[c], &ms, &ap);
    if (rc == PS_OK && e == cudaSuccess && ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
      best_ms = ms;
      best = cands[c];
      best_ap = ap;
    }
  }
  // 2. the schedule, one choice at a time at the best lengths; a choice other
  // than the default is kept only when it is at least 3% faster
  constexpr float kKeep = 0.97f;
  auto try_field = [&](int field, const std::vector<int>& values) {
    for (int val : values) {
      if (e != cudaSuccess || rc != PS_OK || best_ms < 0.f) return;
      std::vector<int> v = best;
      v[field] = val;
      float ms;
      Applies ap;
      rc = trial(v, &ms, &ap);
      if (rc == PS_OK && e == cudaSuccess && ms >= 0.f && ms < kKeep * best_ms) {
        best_ms = ms;
        best = v;
        best_ap = ap;
      }
    }
  };
  const int t0w = p->dtype == PS_F32 ? 16 : 8;
  if (!canonical_order(p)) {
    // x first: the specialised kernels may outrun the extra transforms; the
    // choices below are then tuned for that order
    std::vector<int> v = best;
    v[kXfirst] = 1;
    float ms;
    Applies ap;
    if (e == cudaSuccess && rc == PS_OK && best_ms >= 0.f) {
      rc = trial(v, &ms, &ap);
      if (rc == PS_OK && e == cudaSuccess && ms >= 0.f && ms < kKeep * best_ms) {
        best_ms = ms;
        best = v;
        best_ap = ap;
      }
    }
  }
  if (best_ap.generic) {
    try_field(kTile, {2 * t0w, t0w / 2, t0w / 4});
    try_field(kRadix, {1});
    // then axis by axis: the other tile widths and the other radix split
    for (int j = 0; j < 3; ++j) {
      if (!best_ap.generic_ax[j]) continue;
      const int cur = best[kTile] ? best[kTile] : t0w;
      std::vector<int> tiles;
      for (int t : {2 * t0w, t0w, t0w / 2, t0w / 4})
        if (t != cur) tiles.push_back(t);
      try_field(kTileAx + j, tiles);
      try_field(kRadixAx + j, {best[kRadix] ? 1 : 2});
    }
  }
  if (best_ap.zpipe) try_field(kZtk, {16});
  if (best_ap.chunkable) try_field(kChunks, {2, 4});
  if (best_ap.ypacked) try_field(kYkind, {1, 2});
  {
    // the fused x/y passes: only where the plan's shapes have them
    std::vector<int> v = best;
    v[kXy] = 1;
    float ms;
    Applies ap;
    if (e == cudaSuccess && rc == PS_OK && best_ms >= 0.f) {
      rc = trial(v, &ms, &ap);
      if (rc == PS_OK && e == cudaSuccess && ap.xy && ms >= 0.f && ms < kKeep * best_ms) {
        best_ms = ms;
        best = v;
      }
    }
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
    append_file(key, best);
  }
  return apply_choice(p, best);
}
