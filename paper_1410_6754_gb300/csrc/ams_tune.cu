// Autotuner: picks the plan of a size class -- levels, groups per level r, the
// oversampling factor a, the overpartitioning factor b and the base-case capacity C
// (the tile one block sorts) -- by measurement, as Section 7 tunes a and b.
//
// For (key type, pairs, ceil(log2 n)) it times candidate plans on n synthetic keys of
// two kinds, uniform and duplicate-heavy (P(rank k) ~ 1/k over 2^20 values, scattered
// by SplitMix64), both generated on the device in the given context's scratch; a
// plan's score is the sum of its two times.  Search in two rounds:
//  1. shape: 1, 2 or 3 distribution levels with r = the power of two nearest to
//     (n / t)^(1/levels) for target leaf sizes t = C/2 and C/4, at the default a and
//     b (b = 1 for one level, 4 otherwise);
//  2. parameters of the best shape: (a, b) from the paper's findings -- b = 16 with
//     a = 1.6 log10 n (Section 7.2) and a = 1, b = 64 (the a/b sweep of the appendix)
//     -- plus a = 1 with the default b and b = 16 with a = 1, each where b * r stays
//     within 2048 buckets; and C halved.
// The fastest plan is kept in a process-wide table.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "ams.h"

namespace {

__device__ __forceinline__ uint64_t tune_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Uniform keys, or (skewed) keys of rank floor(2^(20 u)) for uniform u -- P(rank k)
// about 1/k over 2^20 ranks -- scattered through the mixer.
__global__ void k_fill(void* keys, uint64_t* vals, uint64_t n, int ksize, uint64_t seed, int skewed) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t z = tune_mix(seed + (i + 1) * 0x9E3779B97F4A7C15ull);
    if (skewed) {
      const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
      const uint64_t rank = (uint64_t)exp2(20.0 * u);
      z = tune_mix(rank * 0x9E3779B97F4A7C15ull + seed);
    }
    if (ksize == 8) {
      ((uint64_t*)keys)[i] = z;
    } else {
      ((uint32_t*)keys)[i] = (uint32_t)(z >> 32);
    }
    if (vals) vals[i] = i;
  }
}

struct Cand {
  int levels;
  uint32_t r[8];
  uint32_t b;
  uint32_t a;    // 0: the per-segment rule ceil(1.6 log10 n_g)
  uint32_t cap;  // 0: the default base-case capacity
};

std::mutex g_mu;
std::map<std::tuple<int, int, int>, ams_tuned> g_table;

uint32_t pow2_near(double x, uint32_t lo, uint32_t hi) {
  const double l = std::round(std::log2(std::max(x, 1.0)));
  double v = std::pow(2.0, l);
  if (v < lo) v = lo;
  if (v > hi) v = hi;
  return (uint32_t)v;
}

}  // namespace

extern "C" {

AMS_API ams_status ams_tune(void* ctx, uint64_t n, ams_key_type kt, int pairs, void* stream, ams_tuned* out) {
  if (!out || n == 0 || n >= (1ull << 32)) return AMS_ERR_INVALID;
  if (kt != AMS_U32 && kt != AMS_U64 && kt != AMS_F32) return AMS_ERR_INVALID;
  int lg = 0;
  while ((1ull << lg) < n) ++lg;
  const auto key = std::make_tuple((int)kt, pairs ? 1 : 0, lg);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_table.find(key);
    if (it != g_table.end()) {
      *out = it->second;
      return AMS_OK;
    }
  }
  const uint32_t C = ams_default_basecase_cap(kt, pairs);
  std::vector<Cand> shapes;
  if (n <= C) {
    shapes.push_back(Cand{1, {2}, 1, 0, 0});  // no distribution level is launched for n <= C
  } else {
    for (int L = 1; L <= 3; ++L) {
      const uint32_t b = L == 1 ? 1 : 4;
      for (uint32_t t : {C / 2, C / 4}) {
        const double fan = std::pow((double)n / t, 1.0 / L);
        Cand c{L, {}, b, 0, 0};
        const uint32_t r = pow2_near(fan, 2, 2048 / b);
        for (int l = 0; l < L; ++l) c.r[l] = r;
        bool dup = false;
        for (const Cand& o : shapes) dup |= o.levels == c.levels && o.r[0] == c.r[0] && o.b == c.b;
        if (!dup) shapes.push_back(c);
      }
    }
  }
  const size_t w = kt == AMS_U64 ? 8 : 4;
  void *keys = nullptr, *tmp = nullptr;
  uint64_t *vals = nullptr, *vtmp = nullptr;
  const cudaStream_t s = (cudaStream_t)stream;
  ams_status st = AMS_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* keys2 = nullptr;
  if (cudaMalloc(&keys, n * w) != cudaSuccess || cudaMalloc(&keys2, n * w) != cudaSuccess ||
      cudaMalloc(&tmp, n * w) != cudaSuccess ||
      (pairs && (cudaMalloc(&vals, n * 8) != cudaSuccess || cudaMalloc(&vtmp, n * 8) != cudaSuccess))) {
    st = AMS_ERR_OOM;
  } else if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = AMS_ERR_CUDA;
  }
  if (st == AMS_OK) {
    k_fill<<<1024, 256, 0, s>>>(keys, vals, n, (int)w, 0x5EEDull + (uint64_t)lg, 0);
    k_fill<<<1024, 256, 0, s>>>(keys2, nullptr, n, (int)w, 0x5EEDull + (uint64_t)lg, 1);
    if (cudaGetLastError() != cudaSuccess) st = AMS_ERR_CUDA;
  }
  // best of three timed runs (after one warm-up) on each input; score = their sum
  auto score = [&](const Cand& c, float* out_ms) -> ams_status {
    float total = 0.f;
    for (void* in : {keys, keys2}) {
      ams_request rq{};
      rq.keys_in = in;
      rq.keys_out = tmp;
      rq.vals_in = vals;
      rq.vals_out = pairs ? vtmp : nullptr;
      rq.nseg = 1;
      rq.n = n;
      rq.kt = kt;
      rq.levels = c.levels;
      rq.buckets_per_level = c.r;
      rq.opt.overpartition_b = c.b;
      rq.opt.oversample_a = c.a;
      rq.opt.basecase_cap = c.cap;
      float ms = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {
        ams_status e;
        cudaEventRecord(e0, s);
        if ((e = ams_sort_request(ctx, &rq, s)) != AMS_OK) return e;
        cudaEventRecord(e1, s);
        if ((e = ams_context_sync(ctx)) != AMS_OK) return e;
        float t = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
          return AMS_ERR_CUDA;
        if (rep > 0) ms = std::min(ms, t);
      }
      total += ms;
    }
    *out_ms = total;
    return AMS_OK;
  };
  ams_tuned best{};
  best.ms = -1.f;
  uint32_t timed = 0;
  Cand best_c{};
  auto consider = [&](const Cand& c) {
    if (st != AMS_OK) return;
    float ms = 0.f;
    st = score(c, &ms);
    if (st != AMS_OK) return;
    ++timed;
    if (best.ms < 0.f || ms < best.ms) {
      best.levels = c.levels;
      for (int l = 0; l < 8; ++l) best.buckets_per_level[l] = l < c.levels ? c.r[l] : 0;
      best.overpartition_b = c.b;
      best.oversample_a = c.a;
      best.basecase_cap = c.cap;
      best.ms = ms;
      best_c = c;
    }
  };
  for (const Cand& c : shapes) consider(c);
  if (st == AMS_OK && n > C) {
    const Cand shape = best_c;
    std::vector<Cand> params;
    auto with = [&](uint32_t a, uint32_t b, uint32_t cap) {
      Cand c = shape;
      c.a = a;
      c.b = b;
      c.cap = cap;
      if ((uint64_t)b * c.r[0] <= 2048 && (uint64_t)b * c.r[0] >= 2) params.push_back(c);
    };
    with(0, 16, 0);             // b = 16, a = 1.6 log10 n
    with(1, 64, 0);             // a = 1, b = 64
    with(1, shape.b, 0);        // a = 1
    with(1, 16, 0);
    with(0, shape.b, C / 2);    // half the base-case capacity
    for (const Cand& c : params) consider(c);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (keys) cudaFree(keys);
  if (keys2) cudaFree(keys2);
  if (tmp) cudaFree(tmp);
  if (vals) cudaFree(vals);
  if (vtmp) cudaFree(vtmp);
  if (st != AMS_OK) return st;
  best.candidates = timed;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table[key] = best;
  }
  *out = best;
  return AMS_OK;
}

}  // extern "C"
