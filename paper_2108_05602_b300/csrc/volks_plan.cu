// Batch plans: many heterogeneous segments searched by persistent
// launches, optionally replayed from one captured CUDA graph (volks.h,
// volks_plan_*).
//
// Sequence of one run (stream order):
//   per segment   a2-a3 prep launches
//   per round c   zero the peaks of every segment that has a DM chunk c;
//                 per band class (n_f, pad_rate, precision): persistent search over
//                 the class's ranges (dynamic work counter); batched select
//                 and batched match over all ranges of the round.
// A segment's peak/bitmap buffers hold one DM chunk, sized from the plan's
// peak budget, so a round reuses them.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/volks.h"
#include "volks_internal.h"
#include "volks_job.h"
#include "volks_result.h"

struct volks_plan {
  std::vector<std::unique_ptr<vk::SegJob>> jobs;
  std::vector<volks_result*> results;
  int flags = 0;
  int n_rounds = 0;
  // band class (n_f, mode), mode = pad_rate | effective precision << 8
  std::map<std::pair<int, int>, vk::SearchVariant> variant;  // class -> split
  std::map<std::pair<int, int>, int> grid;                   // persistent CTAs
  unsigned long long* d_counters = nullptr;  // n_counters work counters + the error word
  int n_counters = 0;
  bool any_mma = false;
  cudaStream_t work = nullptr;  // capture / autotune stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_stale = true;
  cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
  std::vector<cudaEvent_t> ev_search;  // begin/end pairs
  int n_launch = 0, n_search_launch = 0;
  cudaStream_t last_stream = nullptr;
  bool ran = false;
  long long device_bytes = 0;
};

namespace {

using vk::cuda_fail;
using vk::fail;

std::mutex g_tune_mu;
// autotuned split per (n_f, mode, pad_delay, window mask)
std::map<std::tuple<int, int, int, int>, vk::SearchVariant> g_tuned;

void destroy(volks_plan* p) {
  if (!p) return;
  if (p->last_stream) cudaStreamSynchronize(p->last_stream);
  if (p->work) cudaStreamSynchronize(p->work);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (auto& j : p->jobs) j->release(nullptr);
  if (p->d_counters) cudaFree(p->d_counters);
  for (auto e : p->ev_search) cudaEventDestroy(e);
  if (p->ev_begin) cudaEventDestroy(p->ev_begin);
  if (p->ev_end) cudaEventDestroy(p->ev_end);
  if (p->work) cudaStreamDestroy(p->work);
  for (auto r : p->results) delete r;
  delete p;
}

int class_mode(const vk::SegJob& j) { return j.prm.pad_rate | (j.prec << 8); }
int mode_pad_rate(int mode) { return mode & 0xff; }
int mode_prec(int mode) { return mode >> 8; }
unsigned int* err_word(volks_plan* p) { return reinterpret_cast<unsigned int*>(p->d_counters + p->n_counters); }

struct RangeRef {
  vk::SegJob* job;
  int chunk;
};

// Ranges of round c, grouped by band class.
std::map<std::pair<int, int>, std::vector<RangeRef>> round_classes(volks_plan* p, int c) {
  std::map<std::pair<int, int>, std::vector<RangeRef>> out;
  for (auto& j : p->jobs)
    if (c < j->n_chunks()) out[{j->n_f, class_mode(*j)}].push_back({j.get(), c});
  return out;
}

// Fill batches of at most kMaxDesc ranges; `units` gives a range's work units.
template <class F>
std::vector<vk::Batch> make_batches(const std::vector<RangeRef>& rs, F units) {
  std::vector<vk::Batch> out;
  for (size_t i = 0; i < rs.size(); i += vk::kMaxDesc) {
    vk::Batch b;
    std::memset(&b, 0, sizeof b);
    long long base = 0;
    for (size_t k = i; k < std::min(rs.size(), i + vk::kMaxDesc); ++k) {
      vk::SegDesc d = rs[k].job->desc(rs[k].chunk);
      d.base = base;
      base += units(d);
      b.d[b.n_desc++] = d;
    }
    b.total = base;
    out.push_back(b);
  }
  return out;
}

int n_search_launches(volks_plan* p) {
  int n = 0;
  for (int c = 0; c < p->n_rounds; ++c)
    for (auto& kv : round_classes(p, c)) n += (int)((kv.second.size() + vk::kMaxDesc - 1) / vk::kMaxDesc);
  return n;
}

// Event record that also times graph replays: under capture the record
// becomes an external event node (the flag is invalid outside capture).
cudaError_t record(cudaEvent_t ev, cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &st);
  if (e != cudaSuccess) return e;
  return st == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                             : cudaEventRecord(ev, s);
}

// Enqueue one whole run on stream s (also used under graph capture).
int enqueue_all(volks_plan* p, cudaStream_t s) {
  cudaError_t e;
  p->n_launch = 0;
  p->n_search_launch = 0;
  int counter_i = 0, ev_i = 0;
  if ((e = record(p->ev_begin, s)) != cudaSuccess) return cuda_fail(e, "event");
  if ((e = cudaMemsetAsync(err_word(p), 0, sizeof(unsigned int), s)) != cudaSuccess)
    return cuda_fail(e, "memset error word");
  for (auto& j : p->jobs) {
    if ((e = cudaMemsetAsync(j->d_count, 0, sizeof(unsigned int), s)) != cudaSuccess)
      return cuda_fail(e, "memset count");
    if (j->empty) continue;
    if ((e = j->enqueue_prep(s, &p->n_launch)) != cudaSuccess) return cuda_fail(e, "prep kernels");
  }
  for (int c = 0; c < p->n_rounds; ++c) {
    auto classes = round_classes(p, c);
    std::vector<RangeRef> all;
    for (auto& kv : classes) {
      // every valid segment's key is stored once by the search: no clearing
      for (auto& r : kv.second) all.push_back(r);
    }
    for (auto& kv : classes) {
      const vk::SearchVariant v = p->variant[kv.first];
      auto batches = make_batches(kv.second, [&](const vk::SegDesc& d) { return vk::search_units(d, v); });
      for (auto& b : batches) {
        b.counter = p->d_counters + counter_i++;
        b.err = err_word(p);
        if ((e = cudaMemsetAsync(b.counter, 0, sizeof(unsigned long long), s)) != cudaSuccess)
          return cuda_fail(e, "memset counter");
        if ((e = record(p->ev_search[ev_i++], s)) != cudaSuccess) return cuda_fail(e, "event");
        const int before = p->n_launch;
        e = vk::launch_search_batch(b, v, mode_pad_rate(kv.first.second), mode_prec(kv.first.second),
                                    p->grid[kv.first], s, &p->n_launch);
        if (e != cudaSuccess) return cuda_fail(e, "search kernel");
        p->n_search_launch += p->n_launch - before;
        if ((e = record(p->ev_search[ev_i++], s)) != cudaSuccess) return cuda_fail(e, "event");
      }
    }
    for (auto& b : make_batches(all, [](const vk::SegDesc& d) { return (long long)d.n_bl * d.n_dm * d.n_win; }))
      if ((e = vk::launch_select_batch(b, s, &p->n_launch)) != cudaSuccess) return cuda_fail(e, "select kernel");
    for (auto& b : make_batches(all, [](const vk::SegDesc& d) { return (long long)d.n_bl * d.n_dm; }))
      if ((e = vk::launch_match_batch(b, s, &p->n_launch)) != cudaSuccess) return cuda_fail(e, "match kernel");
  }
  if ((e = record(p->ev_end, s)) != cudaSuccess) return cuda_fail(e, "event");
  return 0;
}

int capture(volks_plan* p) {
  if (p->exec) {
    cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
  }
  if (p->graph) {
    cudaGraphDestroy(p->graph);
    p->graph = nullptr;
  }
  cudaError_t e = cudaStreamBeginCapture(p->work, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
  int rc = enqueue_all(p, p->work);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(p->work, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  p->graph = g;
  e = cudaGraphInstantiate(&p->exec, g, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  p->graph_stale = false;
  return 0;
}

// Time each compiled split of a band class on the first range(s) of round
// 0 and keep the fastest.  The trial runs write peaks that every run
// clears before its search.
int autotune(volks_plan* p, std::pair<int, int> cls, const std::vector<RangeRef>& rs) {
  vk::SearchVariant vs[4];
  const int pr = mode_pad_rate(cls.second), prec = mode_prec(cls.second);
  const int nv = vk::search_variants(cls.first, prec, vs);
  const vk::SegJob& j0 = *rs[0].job;
  const auto key = std::make_tuple(cls.first, cls.second, j0.prm.pad_delay, j0.win_mask);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      p->variant[cls] = it->second;
      return 0;
    }
  }
  if (nv <= 1) {
    p->variant[cls] = vs[0];
    return 0;
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  double best = 1e300;
  vk::SearchVariant best_v = vs[0];
  for (int i = 0; i < nv; ++i) {
    const int occ = vk::search_occupancy(vs[i], pr, prec);
    if (occ <= 0) continue;
    const int grid = occ * vk::sm_count();
    auto batches = make_batches(rs, [&](const vk::SegDesc& d) { return vk::search_units(d, vs[i]); });
    vk::Batch bt = batches[0];
    const long long units = std::min<long long>(bt.total, (long long)grid * 6);
    bt.total = units;
    bt.counter = p->d_counters;
    bt.err = err_word(p);
    float ms_best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      int n = 0;
      cudaMemsetAsync(bt.counter, 0, sizeof(unsigned long long), p->work);
      cudaEventRecord(a, p->work);
      cudaError_t e = vk::launch_search_batch(bt, vs[i], pr, prec, grid, p->work, &n);
      cudaEventRecord(b, p->work);
      if (e != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return cuda_fail(e, "autotune launch");
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0) ms_best = std::min(ms_best, ms);
    }
    // a unit covers a whole tile (all delay residues) in every split
    const double per_point = ms_best / (double)units;
    if (per_point < best) {
      best = per_point;
      best_v = vs[i];
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  p->variant[cls] = best_v;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[key] = best_v;
  return 0;
}

}  // namespace

// Stage times of the plan's last run (volks_result_timing of its results).
int vk_plan_timing(volks_plan* p, volks_timing* t) {
  std::memset(t, 0, sizeof *t);
  if (!p->ran) return 0;
  cudaError_t e = cudaEventSynchronize(p->ev_end);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
  float total = 0.f;
  e = cudaEventElapsedTime(&total, p->ev_begin, p->ev_end);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
  float search = 0.f;
  for (size_t i = 0; i + 1 < p->ev_search.size(); i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->ev_search[i], p->ev_search[i + 1]) == cudaSuccess) search += ms;
  }
  t->ms_search = search;
  t->ms_prep = 0.f;
  t->ms_select = total - search;  // prep + select + match + memsets of the run
  t->n_launches = p->n_launch;
  t->n_search_launches = p->n_search_launch;
  return 0;
}

extern "C" {

int volks_plan_create(const volks_segment* segs, const volks_params* prms, int32_t n, int64_t peak_budget_bytes,
                      int32_t flags, volks_plan** out) {
  if (!out) return fail(VOLKS_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !segs || !prms) return fail(VOLKS_EINVAL, "need n >= 1 segments and parameters");
  if (flags & ~(VOLKS_PLAN_AUTOTUNE | VOLKS_PLAN_GRAPH)) return fail(VOLKS_EINVAL, "unknown plan flags");
  for (int i = 0; i < n; ++i) {
    int rc = vk::validate(&segs[i], &prms[i]);
    if (rc) return fail(rc, "segment %d: %s", i, volks_last_error());
    if ((long long)segs[i].n_bl * segs[i].n_ap > 0) {
      cudaPointerAttributes attr{};
      if (cudaPointerGetAttributes(&attr, segs[i].vis) != cudaSuccess ||
          !(attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return fail(VOLKS_EINVAL, "segment %d: a plan takes device-resident visibilities", i);
      }
      if (segs[i].autos && prms[i].normalize_chan == 1 && !vk::is_device_pointer(segs[i].autos))
        return fail(VOLKS_EINVAL, "segment %d: a plan takes device-resident auto spectra", i);
    }
  }
  volks_plan* p = new (std::nothrow) volks_plan();
  if (!p) return fail(VOLKS_ENOMEM, "host allocation");
  p->flags = flags;
  int rc = 0;
  // jobs with all DMs first, to size the peak buffers
  long long need = 0;
  for (int i = 0; i < n; ++i) {
    p->jobs.emplace_back(new vk::SegJob());
    vk::SegJob& j = *p->jobs.back();
    j.seg_id = i;
    if ((rc = j.init(segs[i], prms[i], 0))) {
      destroy(p);
      return fail(rc, "segment %d: %s", i, volks_last_error());
    }
    if (!j.empty) need += (long long)j.keys_bytes_per_dm() * prms[i].n_dm;
  }
  if (peak_budget_bytes > 0 && need > peak_budget_bytes) {
    for (int i = 0; i < n; ++i) {
      vk::SegJob& j = *p->jobs[i];
      if (j.empty) continue;
      const double share = (double)peak_budget_bytes * ((double)j.keys_bytes_per_dm() * prms[i].n_dm / (double)need);
      const int chunk = std::max(1, (int)(share / (double)j.keys_bytes_per_dm()));
      if ((rc = j.init(segs[i], prms[i], chunk))) {
        destroy(p);
        return fail(rc, "segment %d: %s", i, volks_last_error());
      }
    }
  }
  for (auto& j : p->jobs) {
    p->n_rounds = std::max(p->n_rounds, j->n_chunks());
    p->device_bytes += (long long)j->device_bytes();
  }
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&p->work, cudaStreamNonBlocking)) != cudaSuccess) {
    destroy(p);
    return cuda_fail(e, "cudaStreamCreate");
  }
  for (auto& j : p->jobs) {
    if ((rc = j->alloc(p->work, false)) || (rc = j->stage_input(p->work)) || (rc = j->upload(p->work))) {
      destroy(p);
      return rc;
    }
  }
  // counters: one per search launch
  p->n_counters = std::max(1, n_search_launches(p));
  if ((e = cudaMalloc(&p->d_counters, (p->n_counters + 1) * sizeof(unsigned long long))) != cudaSuccess) {
    destroy(p);
    return cuda_fail(e, "alloc counters");
  }
  if ((e = cudaMemsetAsync(p->d_counters, 0, (p->n_counters + 1) * sizeof(unsigned long long), p->work)) !=
      cudaSuccess) {
    destroy(p);
    return cuda_fail(e, "memset counters");
  }
  p->ev_search.resize(2 * (size_t)n_search_launches(p));
  for (auto& ev : p->ev_search)
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) {
      destroy(p);
      return cuda_fail(e, "cudaEventCreate");
    }
  if ((e = cudaEventCreate(&p->ev_begin)) != cudaSuccess || (e = cudaEventCreate(&p->ev_end)) != cudaSuccess) {
    destroy(p);
    return cuda_fail(e, "cudaEventCreate");
  }
  // work split per band class (autotuned or default) and persistent grid
  for (int c = 0; c < std::min(1, p->n_rounds); ++c)
    for (auto& kv : round_classes(p, c)) {
      if (flags & VOLKS_PLAN_AUTOTUNE) {
        if ((rc = autotune(p, kv.first, kv.second))) {
          destroy(p);
          return rc;
        }
      } else {
        p->variant[kv.first] = vk::default_variant(kv.first.first, mode_prec(kv.first.second), 0);
      }
    }
  for (int c = 0; c < p->n_rounds; ++c)
    for (auto& kv : round_classes(p, c)) {
      if (!p->variant.count(kv.first))
        p->variant[kv.first] = vk::default_variant(kv.first.first, mode_prec(kv.first.second), 0);
      const int occ = vk::search_occupancy(p->variant[kv.first], mode_pad_rate(kv.first.second),
                                           mode_prec(kv.first.second));
      if (mode_prec(kv.first.second) != VOLKS_FP32) p->any_mma = true;
      p->grid[kv.first] = std::max(1, occ) * vk::sm_count();
    }
  if ((e = cudaStreamSynchronize(p->work)) != cudaSuccess) {
    destroy(p);
    return cuda_fail(e, "cudaStreamSynchronize");
  }
  for (int i = 0; i < n; ++i) {
    volks_result* r = new (std::nothrow) volks_result();
    if (!r) {
      destroy(p);
      return fail(VOLKS_ENOMEM, "host allocation");
    }
    r->job = p->jobs[i].get();
    r->borrowed = true;
    r->plan = p;
    if (p->any_mma) r->d_err = err_word(p);
    r->stream = p->work;
    r->synced = true;
    p->results.push_back(r);
  }
  *out = p;
  return 0;
}

int volks_plan_run(volks_plan* p, const void* const* vis, void* cuda_stream) {
  if (!p) return fail(VOLKS_EINVAL, "NULL plan");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (vis) {
    for (size_t i = 0; i < p->jobs.size(); ++i) {
      vk::SegJob& j = *p->jobs[i];
      if (j.empty || vis[i] == j.d_vis) continue;
      cudaPointerAttributes attr{};
      if (!vis[i] || cudaPointerGetAttributes(&attr, vis[i]) != cudaSuccess ||
          !(attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return fail(VOLKS_EINVAL, "segment %zu: a plan takes device-resident visibilities", i);
      }
      j.d_vis = static_cast<const float2*>(vis[i]);
      j.seg.vis = vis[i];
      p->graph_stale = true;
    }
  }
  // the previous run's results must not be read while this one overwrites them
  if (p->last_stream && p->last_stream != s) {
    cudaError_t e = cudaStreamSynchronize(p->last_stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  }
  int rc = 0;
  if (p->flags & VOLKS_PLAN_GRAPH) {
    if (p->graph_stale && (rc = capture(p))) return rc;
    cudaError_t e = cudaGraphLaunch(p->exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  } else {
    if ((rc = enqueue_all(p, s))) return rc;
  }
  p->last_stream = s;
  p->ran = true;
  for (auto r : p->results) {
    r->stream = s;
    r->synced = false;
    r->have_cands = false;
    r->cands.clear();
  }
  return 0;
}

int volks_plan_result(volks_plan* p, int32_t i, volks_result** res) {
  if (!p || !res) return fail(VOLKS_EINVAL, "NULL argument");
  if (i < 0 || i >= (int)p->results.size()) return fail(VOLKS_EINVAL, "segment index %d out of range", i);
  *res = p->results[i];
  return 0;
}

int volks_plan_timing(volks_plan* p, volks_timing* t) {
  if (!p || !t) return fail(VOLKS_EINVAL, "NULL argument");
  return vk_plan_timing(p, t);
}

int volks_plan_info(volks_plan* p, int32_t* n_rounds, int64_t* device_bytes, int32_t* n_search_launches_per_run) {
  if (!p) return fail(VOLKS_EINVAL, "NULL plan");
  if (n_rounds) *n_rounds = p->n_rounds;
  if (device_bytes) *device_bytes = p->device_bytes;
  if (n_search_launches_per_run) *n_search_launches_per_run = n_search_launches(p);
  return 0;
}

void volks_plan_free(volks_plan* p) { destroy(p); }

int volks_search_batch(const volks_segment* segs, const volks_params* prms, int32_t n, void* cuda_stream,
                       volks_plan** out) {
  if (!out) return fail(VOLKS_EINVAL, "out is NULL");
  *out = nullptr;
  volks_plan* p = nullptr;
  int rc = volks_plan_create(segs, prms, n, 0, 0, &p);
  if (rc) return rc;
  rc = volks_plan_run(p, nullptr, cuda_stream);
  if (rc) {
    volks_plan_free(p);
    return rc;
  }
  *out = p;
  return 0;
}

}  // extern "C"
