// Continuous-batching request server (volks_server_* in include/volks.h).
//
// Requests (scan segments) are queued by volks_server_submit.  A scheduler
// thread admits them in arrival order while a slot (CUDA stream) is free
// and their device scratch fits the HBM budget, and enqueues each admitted
// search on its slot's stream, so requests that arrive while others run
// overlap on the device.  A completion thread polls the admitted searches,
// gathers each finished one's candidates (window match on the device,
// cross-baseline match on the host), releases its budget and slot and
// records its latency.
//
// Consecutive segments of one stream (stream_id >= 0) keep a
// device-resident halo: the last H APs of each segment (H = the largest
// dispersion shift of the stream's DM grid) are prepended to the next
// segment, so a pulse that crosses a segment boundary is searched whole.
// Segments of one stream are searched one after another in submission
// order.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/volks.h"
#include "volks_internal.h"
#include "volks_job.h"
#include "volks_result.h"

namespace {

using vk::cuda_fail;
using vk::fail;
using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  volks_segment seg{};
  volks_params prm{};
  std::vector<double> cal;
  std::vector<int32_t> bl_st;
  int64_t stream_id = -1;
  Clock::time_point t_submit, t_admit, t_done;
  int64_t bytes = 0;
  int status = 1;  // 1 queued, 2 running, 0 done, < 0 failed (VOLKS_E*)
  int slot = -1;
  int64_t ap_offset = 0;
  long long trials = 0;
  int halo_H = 0;  // stream requests: halo length
  volks_result* res = nullptr;
  void* ext = nullptr;  // stream requests: halo + segment (device), owned
  std::vector<volks_candidate> cands;
  std::string err;
};

struct Halo {
  int n_bl = 0, n_f = 0, H = 0;
  bool valid = false;
  void* buf = nullptr;  // [n_bl][H][n_f] complex64, device
  int64_t next_ap = 0;  // stream AP index of the next segment's first AP
  bool busy = false;    // a segment of this stream is admitted and not done
};

long long trial_count(const vk::SegJob& j) {
  long long n = 0;
  for (int d = 0; d < j.prm.n_dm; ++d) {
    const int nv = std::max(0, j.nvalid[d]);
    for (int i = 0; i < j.prm.n_win; ++i) n += vk::seg_count(nv, j.win_log[i], j.slide ? 1 : 0);
  }
  return n * j.seg.n_bl;
}

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct volks_server {
  volks_server_config cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  std::vector<std::shared_ptr<Request>> running;
  std::vector<cudaStream_t> streams;
  std::vector<char> slot_busy;
  std::map<int64_t, Halo> halos;
  int64_t bytes_in_use = 0, peak_bytes = 0;
  int peak_inflight = 0;
  uint64_t next_id = 1;
  int64_t admissions = 0;
  bool stop = false;
  std::thread sched, done;
  std::vector<double> lat_ms;
  long long trials_done = 0;
  Clock::time_point t_first, t_last;
  bool any = false;
  int64_t submitted = 0, completed = 0, failed = 0;
};

namespace {

// Enqueue the search of an admitted request on its slot's stream.  Called
// by the scheduler thread without the lock (the request is owned by it
// until its status leaves 2 only through the completion thread).
int launch(volks_server* S, Request& r, Halo* h) {
  cudaStream_t st = S->streams[r.slot];
  volks_segment seg = r.seg;
  seg.cal = r.cal.empty() ? nullptr : r.cal.data();
  seg.bl_st = r.bl_st.empty() ? nullptr : r.bl_st.data();
  if (S->cfg.fail_every > 0 && (S->admissions % S->cfg.fail_every) == 0)
    return fail(VOLKS_ENOMEM, "injected allocation failure (fail_every = %d)", S->cfg.fail_every);
  if (h) {
    // ext = [halo (H APs, if valid) | segment]; afterwards the last H APs of
    // ext become the halo of the stream's next segment
    const int H = h->H, n_bl = seg.n_bl, n_f = seg.n_if * seg.n_chan;
    const int pre = h->valid ? H : 0;
    const int n_ext = pre + seg.n_ap;
    const size_t row = (size_t)n_f * sizeof(float2);
    cudaError_t e = cudaMallocAsync(&r.ext, (size_t)n_bl * n_ext * row, st);
    if (e != cudaSuccess) return cuda_fail(e, "alloc stream input");
    if (pre)
      if ((e = cudaMemcpy2DAsync(r.ext, n_ext * row, h->buf, (size_t)H * row, (size_t)H * row, n_bl,
                                 cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "copy halo");
    if ((e = cudaMemcpy2DAsync(static_cast<char*>(r.ext) + pre * row, n_ext * row, seg.vis, seg.n_ap * row,
                               seg.n_ap * row, n_bl, cudaMemcpyDefault, st)) != cudaSuccess)
      return cuda_fail(e, "copy segment");
    r.ap_offset = h->next_ap - pre;
    seg.vis = r.ext;
    seg.n_ap = n_ext;
    int rc = volks_search_segment(&seg, &r.prm, st, &r.res);
    if (rc) return rc;
    if ((e = cudaMemcpy2DAsync(h->buf, (size_t)H * row, static_cast<char*>(r.ext) + (size_t)(n_ext - H) * row,
                               n_ext * row, (size_t)H * row, n_bl, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "save halo");
    return 0;
  }
  return volks_search_segment(&seg, &r.prm, st, &r.res);
}

void scheduler(volks_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    std::shared_ptr<Request> pick;
    int slot = -1;
    Halo* h = nullptr;
    S->cv_sched.wait(lk, [&] {
      if (S->stop) return true;
      slot = -1;
      for (int i = 0; i < (int)S->slot_busy.size(); ++i)
        if (!S->slot_busy[i]) {
          slot = i;
          break;
        }
      if (slot < 0) return false;
      // arrival order; a request waiting for its stream's previous segment
      // is skipped, one that does not fit the budget blocks the queue
      for (auto& q : S->pending) {
        if (q->stream_id >= 0 && S->halos[q->stream_id].busy) continue;
        if (S->bytes_in_use + q->bytes > S->cfg.hbm_budget_bytes) return false;
        pick = q;
        return true;
      }
      return false;
    });
    if (S->stop) return;
    S->pending.erase(std::find(S->pending.begin(), S->pending.end(), pick));
    pick->slot = slot;
    pick->status = 2;
    pick->t_admit = Clock::now();
    S->slot_busy[slot] = 1;
    S->bytes_in_use += pick->bytes;
    S->peak_bytes = std::max(S->peak_bytes, S->bytes_in_use);
    if (pick->stream_id >= 0) {
      h = &S->halos[pick->stream_id];
      h->busy = true;
    }
    ++S->admissions;
    int n_run = 0;
    for (auto& q : S->running) n_run += q->status == 2;
    S->peak_inflight = std::max(S->peak_inflight, n_run + 1);
    lk.unlock();
    const int rc = launch(S, *pick, h);
    lk.lock();
    if (rc) {
      pick->err = volks_last_error();
      pick->status = rc;  // the completion thread retires it
    } else if (h) {
      h->valid = true;
      h->next_ap += pick->seg.n_ap;
    }
    S->running.push_back(pick);
    S->cv_done.notify_all();
  }
}

// Retire finished requests (polling, so none waits behind an older one).
void completer(volks_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_done.wait_for(lk, std::chrono::microseconds(200), [&] { return S->stop || !S->running.empty(); });
    if (S->stop && S->running.empty()) return;
    std::vector<std::shared_ptr<Request>> ready;
    for (auto& q : S->running) {
      if (q->status < 0 || !q->res) {
        ready.push_back(q);
        continue;
      }
      // the search's last event; the halo save follows it on the stream
      if (cudaStreamQuery(S->streams[q->slot]) == cudaSuccess) ready.push_back(q);
    }
    if (ready.empty()) continue;
    for (auto& q : ready) S->running.erase(std::find(S->running.begin(), S->running.end(), q));
    lk.unlock();
    for (auto& q : ready) {
      if (q->status == 2) {
        size_t n = 0;
        int rc = volks_candidates(q->res, nullptr, 0, &n);
        if (!rc) {
          q->cands.resize(n);
          rc = volks_candidates(q->res, q->cands.data(), n, &n);
        }
        if (!rc) q->trials = trial_count(*q->res->job);
        if (rc) {
          q->status = rc;
          q->err = volks_last_error();
        }
      }
      cudaStream_t st = q->slot >= 0 ? S->streams[q->slot] : nullptr;
      if (q->res) volks_free(q->res);
      q->res = nullptr;
      if (q->ext) cudaFreeAsync(q->ext, st);
      q->ext = nullptr;
      q->t_done = Clock::now();
    }
    lk.lock();
    for (auto& q : ready) {
      if (q->slot >= 0) S->slot_busy[q->slot] = 0;
      S->bytes_in_use -= q->bytes;
      if (q->stream_id >= 0) S->halos[q->stream_id].busy = false;
      if (q->status == 2) {
        q->status = 0;
        ++S->completed;
        S->lat_ms.push_back(ms_between(q->t_submit, q->t_done));
        S->trials_done += q->trials;
        S->t_last = q->t_done;
      } else {
        ++S->failed;
      }
    }
    S->cv_done.notify_all();
    S->cv_sched.notify_all();
  }
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double x = p * (v.size() - 1);
  const size_t i = (size_t)x;
  const double f = x - i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

int volks_server_create(const volks_server_config* cfg, volks_server** out) {
  if (!out || !cfg) return fail(VOLKS_EINVAL, "NULL argument");
  *out = nullptr;
  if (cfg->max_inflight < 1 || cfg->max_inflight > 64) return fail(VOLKS_EINVAL, "max_inflight must be 1..64");
  if (cfg->hbm_budget_bytes <= 0) return fail(VOLKS_EINVAL, "hbm_budget_bytes must be > 0");
  if (cfg->fail_every < 0) return fail(VOLKS_EINVAL, "fail_every must be >= 0");
  volks_server* S = new (std::nothrow) volks_server();
  if (!S) return fail(VOLKS_ENOMEM, "host allocation");
  S->cfg = *cfg;
  cudaError_t e = cudaGetDevice(&S->device);
  if (e != cudaSuccess) {
    delete S;
    return cuda_fail(e, "cudaGetDevice");
  }
  S->streams.resize(cfg->max_inflight);
  S->slot_busy.assign(cfg->max_inflight, 0);
  for (auto& s : S->streams)
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) {
      for (auto& x : S->streams)
        if (x) cudaStreamDestroy(x);
      delete S;
      return cuda_fail(e, "cudaStreamCreate");
    }
  S->sched = std::thread(scheduler, S);
  S->done = std::thread(completer, S);
  *out = S;
  return 0;
}

int volks_server_submit(volks_server* S, const volks_segment* seg, const volks_params* prm, int64_t stream_id,
                        uint64_t* id) {
  if (!S || !id) return fail(VOLKS_EINVAL, "NULL argument");
  int rc = vk::validate(seg, prm);
  if (rc) return rc;
  auto r = std::make_shared<Request>();
  r->seg = *seg;
  r->prm = *prm;
  r->stream_id = stream_id;
  const size_t n_pol = seg->n_pol == 2 ? 2 : 1;
  if (seg->cal) r->cal.assign(seg->cal, seg->cal + n_pol * seg->n_bl * seg->n_if * 2);
  if (seg->autos && prm->normalize_chan == 1 && seg->bl_st)
    r->bl_st.assign(seg->bl_st, seg->bl_st + (size_t)seg->n_bl * 2);
  if (stream_id >= 0 && (n_pol > 1 || seg->autos))
    return fail(VOLKS_EINVAL, "chained segments (stream_id >= 0) take one polarisation product and no auto spectra");
  // device bytes of the search (plus a copy of host input, plus the halo)
  vk::SegJob j;
  if ((rc = j.init(*seg, *prm, 0))) return rc;
  r->bytes = (int64_t)j.device_bytes();
  const size_t vis_bytes = (size_t)seg->n_bl * seg->n_ap * j.n_f * sizeof(float2);
  if (!vk::is_device_pointer(seg->vis)) r->bytes += (int64_t)(n_pol * vis_bytes);
  if (j.use_autos && !vk::is_device_pointer(seg->autos))
    r->bytes += (int64_t)(j.input_bytes() - n_pol * vis_bytes);
  std::unique_lock<std::mutex> lk(S->mu);
  if (stream_id >= 0) {
    int H = 0;
    for (int d = 0; d < prm->n_dm; ++d) H = std::max(H, seg->n_ap - j.nvalid[d]);
    Halo& h = S->halos[stream_id];
    if (!h.buf) {
      h.n_bl = seg->n_bl;
      h.n_f = j.n_f;
      h.H = std::max(1, H);
      cudaError_t e = cudaMalloc(&h.buf, (size_t)h.n_bl * h.H * h.n_f * sizeof(float2));
      if (e != cudaSuccess) {
        S->halos.erase(stream_id);
        return cuda_fail(e, "alloc halo");
      }
    }
    if (h.n_bl != seg->n_bl || h.n_f != j.n_f || H > h.H || seg->n_ap < h.H)
      return fail(VOLKS_EINVAL, "stream %lld: segments need %d baselines, %d points, >= %d APs and no "
                  "larger dispersion sweep than the first", (long long)stream_id, h.n_bl, h.n_f, h.H);
    r->halo_H = h.H;
    // the extended input: halo + segment, plus its normalised copy
    r->bytes += 2 * (int64_t)seg->n_bl * h.H * j.n_f * (int64_t)sizeof(float2) + (int64_t)vis_bytes;
  }
  if (r->bytes > S->cfg.hbm_budget_bytes)
    return fail(VOLKS_ENOMEM, "request needs %lld device bytes, the budget is %lld", (long long)r->bytes,
                (long long)S->cfg.hbm_budget_bytes);
  r->id = S->next_id++;
  r->t_submit = Clock::now();
  if (!S->any) {
    S->t_first = r->t_submit;
    S->any = true;
  }
  ++S->submitted;
  S->all[r->id] = r;
  S->pending.push_back(r);
  *id = r->id;
  S->cv_sched.notify_all();
  return 0;
}

int volks_server_wait(volks_server* S, uint64_t id, int32_t timeout_ms, volks_candidate* buf, size_t cap,
                      size_t* n_total, volks_request_info* info) {
  if (!S || !n_total) return fail(VOLKS_EINVAL, "NULL argument");
  if (cap > 0 && !buf) return fail(VOLKS_EINVAL, "NULL buffer with cap > 0");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return fail(VOLKS_EINVAL, "unknown or already collected request %llu", (unsigned long long)id);
  std::shared_ptr<Request> r = it->second;
  const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
  if (!S->cv_done.wait_until(lk, deadline, [&] { return r->status <= 0; }))
    return fail(VOLKS_ETIMEOUT, "request %llu not finished within %d ms", (unsigned long long)id, timeout_ms);
  if (info) {
    std::memset(info, 0, sizeof *info);
    info->status = r->status;
    info->queue_ms = ms_between(r->t_submit, r->t_admit);
    info->latency_ms = ms_between(r->t_submit, r->t_done);
    info->device_bytes = r->bytes;
    info->ap_offset = r->ap_offset;
    info->trials = r->trials;
  }
  S->all.erase(it);
  if (r->status < 0) return fail(r->status, "request %llu failed: %s", (unsigned long long)id, r->err.c_str());
  *n_total = r->cands.size();
  const size_t n = std::min(cap, r->cands.size());
  if (n) std::memcpy(buf, r->cands.data(), n * sizeof(volks_candidate));
  return 0;
}

int volks_server_get_stats(volks_server* S, volks_server_stats* st) {
  if (!S || !st) return fail(VOLKS_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(st, 0, sizeof *st);
  st->submitted = S->submitted;
  st->completed = S->completed;
  st->failed = S->failed;
  st->queued = (int32_t)S->pending.size();
  int n_run = 0;
  for (auto& q : S->running) n_run += q->status == 2;
  st->inflight = n_run;
  st->peak_inflight = S->peak_inflight;
  st->bytes_in_use = S->bytes_in_use;
  st->peak_bytes = S->peak_bytes;
  st->p50_ms = percentile(S->lat_ms, 0.50);
  st->p99_ms = percentile(S->lat_ms, 0.99);
  double sum = 0.0;
  for (double x : S->lat_ms) sum += x;
  st->mean_ms = S->lat_ms.empty() ? 0.0 : sum / S->lat_ms.size();
  st->trials = S->trials_done;
  const double span = S->completed ? ms_between(S->t_first, S->t_last) / 1e3 : 0.0;
  st->trials_per_s = span > 0 ? S->trials_done / span : 0.0;
  return 0;
}

int volks_server_drain(volks_server* S, int32_t timeout_ms) {
  if (!S) return fail(VOLKS_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
  if (!S->cv_done.wait_until(lk, deadline, [&] { return S->pending.empty() && S->running.empty(); }))
    return fail(VOLKS_ETIMEOUT, "server not drained within %d ms", timeout_ms);
  return 0;
}

void volks_server_free(volks_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_sched.notify_all();
  S->cv_done.notify_all();
  if (S->sched.joinable()) S->sched.join();
  if (S->done.joinable()) S->done.join();  // retires what is still running
  for (auto& s : S->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (auto& kv : S->halos)
    if (kv.second.buf) cudaFree(kv.second.buf);
  delete S;
}

}  // extern "C"
