// Serving loop: continuous batching of deblur requests against device-resident factored
// Hessian sets (the Hessians of Algorithm 2 are built once and reused for every source and
// every request; the deblur of one request is eq. Qsystemfreq solved per frequency for all its
// sources, with the inverse transform back to time).
//
// Requests (residual gathers of any source count and trace length) are queued by
// egh_server_submit.  A worker thread admits them in arrival order into free slots (one CUDA
// stream each) as long as their device buffers fit in an arena reserved at creation (the HBM
// budget); queued requests for the same Hessian set are packed into one batch that shares the
// per-frequency solve (the spectra of each request occupy their own columns).  Each batch runs
// H2D copy -> forward transform -> solve (-> refinement) -> synthesis -> D2H copy on its stream;
// batches in different slots overlap on the device.  A host callback on the stream marks the
// batch's requests done, releases its arena blocks and wakes the worker, which admits the next
// requests at once.  No device allocation happens after creation.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "egh.h"
#include "egh_internal.cuh"

using namespace egh;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device region (offsets aligned to 256 bytes).
class Arena {
 public:
  void reset(size_t bytes) {
    free_.clear();
    free_[0] = bytes;
    total_ = bytes;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t total() const { return total_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t total_ = 0, used_ = 0, peak_ = 0;
};

struct HSet {
  int nrec = 0, nf = 0, tw_len = 0;
  float2 *Qh = nullptr, *Lh = nullptr, *tw = nullptr;
  float2* Wh = nullptr;  // mixed precision: W = L^{-1}
  float2* Ph = nullptr;  // mixed precision: Q^{-1} = W^H W
  int* kref = nullptr;   // mixed precision: frequencies whose solves are refined (device list)
  int nref = 0;
  unsigned char* twt = nullptr;  // tensor-core transform twiddle tiles (tw_len levels)
  unsigned char* tws = nullptr;  // tensor-core synthesis twiddle tiles (tw_len samples)
  float* w = nullptr;
};

struct Request {
  long long id = 0;
  int set = 0, ns = 0, nt_d = 0;
  const float* resid = nullptr;
  float* mult = nullptr;
  double t_submit = 0, t_done = 0;
  bool done = false;
  egh_status status = EGH_OK;  // EGH_ETIMEOUT: a bounded device wait of its batch ran out
  std::string msg;             // why the request failed
  size_t off_in = 0, off_out = 0, bytes = 0;
};

struct Server;

struct Batch {
  Server* sv = nullptr;
  int slot = -1;
  std::vector<Request*> reqs;
  size_t off_d = 0, bytes_d = 0;
};

struct Server {
  int dev = 0;
  int prec = EGH_PREC_FP32;
  int nslots = 0, max_batch = 0;
  char* arena_base = nullptr;
  int* d_err = nullptr;  // [slots] device flags, set by a kernel whose bounded wait ran out
  int* h_err = nullptr;  // [slots] pinned host copies, read when a batch completes
  int expire = 0;        // test hook: batches whose forward transform has one wait run out
  long long device_timeouts = 0;  // batches with an expired wait since the last drain
  Arena arena;
  std::vector<HSet> sets;
  std::vector<cudaStream_t> streams;
  std::vector<bool> slot_busy;
  std::deque<Request*> queue;
  std::map<long long, Request*> reqs;
  long long next_id = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  bool held = false;  // admission paused by egh_server_hold
  std::string worker_error;
  int in_flight = 0, peak_in_flight = 0;
  // statistics
  long long submitted = 0, completed = 0, rejected = 0, sources_done = 0, batches = 0;
  std::vector<double> latencies;
  double t_first = 0, t_last = 0;
  std::string err;
};

egh_status fail(Server* sv, egh_status s, const std::string& msg) {
  if (sv)
    sv->err = msg;
  else
    set_context_free_error(msg);
  return s;
}

size_t d_bytes(const Server* sv, const HSet& h, int ns_total) {
  return (size_t)h.nf * h.nrec * ns_total * sizeof(float2) * (prec_mixed(sv->prec) ? 3 : 1);
}

size_t trace_bytes(const HSet& h, int ns, int nt_d) {
  return (size_t)ns * h.nrec * nt_d * sizeof(float);
}

// Host callback at the end of a batch's stream work: requests done, arena blocks released.
void CUDART_CB batch_done(void* p) {
  Batch* b = static_cast<Batch*>(p);
  Server* sv = b->sv;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    const double t = now_s();
    // the slot's error flag was copied to the host just before this callback
    const bool expired = sv->h_err[b->slot] != 0;
    if (expired) ++sv->device_timeouts;
    for (Request* r : b->reqs) {
      r->t_done = t;
      r->done = true;
      if (expired) {
        r->status = EGH_ETIMEOUT;
        r->msg = "a bounded device wait ran out in this request's batch; its multipliers are not valid";
      }
      sv->arena.release(r->off_in, r->bytes);
      sv->arena.release(r->off_out, r->bytes);
      sv->latencies.push_back(t - r->t_submit);
      sv->sources_done += r->ns;
      ++sv->completed;
    }
    sv->t_last = t;
    sv->arena.release(b->off_d, b->bytes_d);
    sv->slot_busy[b->slot] = false;
    --sv->in_flight;
  }
  sv->cv_work.notify_all();
  sv->cv_done.notify_all();
  delete b;
}

// Enqueues one batch on its slot's stream (called by the worker with the lock released).
cudaError_t run_batch(Server* sv, Batch* b, const HSet& h, int expire) {
  cudaStream_t st = sv->streams[b->slot];
  int* err = sv->d_err + b->slot;
  int ld = 0;
  for (Request* r : b->reqs) ld += r->ns;
  float2* D = reinterpret_cast<float2*>(sv->arena_base + b->off_d);
  const size_t dsz = (size_t)h.nf * h.nrec * ld;
  cudaError_t e;
  if ((e = cudaMemsetAsync(err, 0, sizeof(int), st))) return e;
  int s0 = 0;
  for (Request* r : b->reqs) {
    float* din = reinterpret_cast<float*>(sv->arena_base + r->off_in);
    if ((e = cudaMemcpyAsync(din, r->resid, r->bytes, cudaMemcpyHostToDevice, st))) return e;
    if ((e = launch_trace_dft(din, r->ns * h.nrec, r->nt_d, h.nf, h.nrec, ld, s0, D, st,
                              h.twt, err, s0 == 0 ? expire : 0, true)))
      return e;
    s0 += r->ns;
  }
  float2* Xs = D;  // the solutions the synthesis reads
  if (prec_mixed(sv->prec)) {
    // Y = Q^{-1} D on the tensor cores; at the frequencies whose condition bound asks for it, the
    // residual R = D - Q Y to FP64-class accuracy and the correction Y += Q^{-1} R
    float2* Y = D + dsz;
    float2* R = D + 2 * dsz;
    if ((e = launch_cmm_tc(h.Ph, h.nrec, h.nf, D, ld, Y, nullptr, err, st))) return e;
    if (h.nref > 0) {
      if ((e = launch_resid(h.Qh, h.nrec, h.nref, Y, D, ld, R, sv->prec == EGH_PREC_MIXED_FP64, st,
                            h.kref)))
        return e;
      if ((e = launch_cmm_tc(h.Ph, h.nrec, h.nref, R, ld, D, h.kref, err, st))) return e;
      if ((e = launch_add_correction(Y, D, (long long)h.nrec * ld, h.nref, st, h.kref))) return e;
    }
    Xs = Y;
  } else {
    if ((e = launch_trsm(h.Lh, h.nrec, h.nf, D, ld, st))) return e;
  }
  s0 = 0;
  for (Request* r : b->reqs) {
    float* dout = reinterpret_cast<float*>(sv->arena_base + r->off_out);
    // the request's residual buffer, read by its forward transform above, holds the synthesis
    // operand images when it is large enough
    float* din = reinterpret_cast<float*>(sv->arena_base + r->off_in);
    if ((e = launch_synth(Xs, h.nrec, r->ns, ld, s0, h.nf, h.w, h.tw, r->nt_d, dout, st, h.tws,
                          err, true, reinterpret_cast<unsigned char*>(din), r->bytes)))
      return e;
    if ((e = cudaMemcpyAsync(r->mult, dout, r->bytes, cudaMemcpyDeviceToHost, st))) return e;
    s0 += r->ns;
  }
  if ((e = cudaMemcpyAsync(sv->h_err + b->slot, err, sizeof(int), cudaMemcpyDeviceToHost, st)))
    return e;
  return cudaLaunchHostFunc(st, batch_done, b);
}

// A batch whose work could not be enqueued: its requests fail with EGH_ECUDA, and its memory and
// slot are released once whatever was enqueued on its stream has finished (caller holds the lock).
void batch_failed(Server* sv, Batch* b, const std::string& msg) {
  cudaStreamSynchronize(sv->streams[b->slot]);
  cudaGetLastError();
  const double t = now_s();
  for (Request* r : b->reqs) {
    r->t_done = t;
    r->done = true;
    r->status = EGH_ECUDA;
    r->msg = msg;
    sv->arena.release(r->off_in, r->bytes);
    sv->arena.release(r->off_out, r->bytes);
  }
  sv->arena.release(b->off_d, b->bytes_d);
  sv->slot_busy[b->slot] = false;
  --sv->in_flight;
  delete b;
}

// Worker: admits queued requests in arrival order into free slots while their buffers fit.
void worker_loop(Server* sv) {
  cudaSetDevice(sv->dev);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    // wake for work (a queued request and a free slot) or to leave (stopping with nothing queued)
    sv->cv_work.wait(lk, [&] {
      if (!sv->worker_error.empty()) return true;
      if (sv->queue.empty()) return sv->stop;
      if (sv->held && !sv->stop) return false;
      for (bool b : sv->slot_busy)
        if (!b) return true;
      return false;
    });
    if (!sv->worker_error.empty() || (sv->stop && sv->queue.empty())) break;
    int slot = -1;
    for (int i = 0; i < sv->nslots; ++i)
      if (!sv->slot_busy[i]) {
        slot = i;
        break;
      }
    if (slot < 0) continue;
    // the head request and the following requests of the same set, up to the batch limit
    Request* head = sv->queue.front();
    const HSet& h = sv->sets[head->set];
    std::vector<Request*> pick;
    int ns_total = 0;
    for (Request* r : sv->queue) {
      if (r->set != head->set) continue;
      if (!pick.empty() && ns_total + r->ns > sv->max_batch) break;
      pick.push_back(r);
      ns_total += r->ns;
    }
    // fit the buffers; drop requests from the tail of the pick until they fit
    Batch* b = new Batch();
    b->sv = sv;
    b->slot = slot;
    bool ok = false;
    while (!pick.empty()) {
      ns_total = 0;
      for (Request* r : pick) ns_total += r->ns;
      size_t off_d = 0;
      const size_t bd = d_bytes(sv, h, ns_total);
      if (sv->arena.alloc(bd, &off_d)) {
        std::vector<std::pair<size_t, size_t>> got;
        bool all = true;
        for (Request* r : pick) {
          size_t a = 0, c = 0;
          if (!sv->arena.alloc(r->bytes, &a)) {
            all = false;
            break;
          }
          if (!sv->arena.alloc(r->bytes, &c)) {
            sv->arena.release(a, r->bytes);
            all = false;
            break;
          }
          r->off_in = a;
          r->off_out = c;
          got.emplace_back(a, c);
        }
        if (all) {
          b->off_d = off_d;
          b->bytes_d = bd;
          ok = true;
          break;
        }
        for (size_t i = 0; i < got.size(); ++i) {
          sv->arena.release(got[i].first, pick[i]->bytes);
          sv->arena.release(got[i].second, pick[i]->bytes);
        }
        sv->arena.release(off_d, bd);
      }
      pick.pop_back();
    }
    if (!ok) {
      // nothing fits now: wait until a batch in flight releases memory
      delete b;
      if (sv->in_flight == 0) {
        // cannot happen (every request fits the budget alone, checked at submission)
        sv->worker_error = "a request does not fit the arena with nothing in flight";
        Request* r = sv->queue.front();
        sv->queue.pop_front();
        r->done = true;
        ++sv->rejected;
        sv->cv_done.notify_all();
        continue;
      }
      sv->cv_work.wait(lk);
      continue;
    }
    for (Request* r : pick) sv->queue.erase(std::find(sv->queue.begin(), sv->queue.end(), r));
    b->reqs = pick;
    sv->slot_busy[slot] = true;
    ++sv->in_flight;
    sv->peak_in_flight = std::max(sv->peak_in_flight, sv->in_flight);
    ++sv->batches;
    const HSet hs = h;  // the set list may grow while the lock is released
    const int expire = sv->expire > 0 ? 1 : 0;
    if (expire) --sv->expire;
    lk.unlock();
    const cudaError_t e = run_batch(sv, b, hs, expire);
    lk.lock();
    if (e != cudaSuccess) {
      // the batch's requests fail; queued requests fail at egh_server_wait (the server stops)
      sv->worker_error = std::string("batch launch: ") + cudaGetErrorString(e);
      batch_failed(sv, b, sv->worker_error);
      sv->stop = true;
      sv->cv_done.notify_all();
      break;
    }
  }
}

}  // namespace

struct egh_server : Server {};

extern "C" {

egh_status egh_server_create(const egh_server_config* cfg, egh_server** out) {
  if (!out || !cfg) return fail(nullptr, EGH_EINVAL, "NULL argument");
  *out = nullptr;
  for (int v : cfg->reserved)
    if (v != 0) return fail(nullptr, EGH_EINVAL, "reserved server fields must be zero");
  if (cfg->hbm_budget_bytes < (1 << 20)) return fail(nullptr, EGH_EINVAL, "hbm_budget_bytes must be >= 1 MiB");
  if (cfg->slots < 1 || cfg->slots > 16) return fail(nullptr, EGH_EINVAL, "slots must be in 1..16");
  if (cfg->max_batch_sources < 1) return fail(nullptr, EGH_EINVAL, "max_batch_sources must be >= 1");
  if (cfg->precision != EGH_PREC_FP32 && !prec_mixed(cfg->precision))
    return fail(nullptr, EGH_EINVAL, "unknown precision");
  egh_server* sv = new (std::nothrow) egh_server();
  if (!sv) return fail(nullptr, EGH_ENOMEM, "host allocation failed");
  cudaGetDevice(&sv->dev);
  sv->prec = cfg->precision;
  sv->nslots = cfg->slots;
  sv->max_batch = cfg->max_batch_sources;
  cudaError_t e = cudaMalloc(&sv->arena_base, (size_t)cfg->hbm_budget_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete sv;
    return fail(nullptr, EGH_ENOMEM, std::string("arena: ") + cudaGetErrorString(e));
  }
  const size_t flag_bytes = sizeof(int) * (size_t)cfg->slots;
  if ((e = cudaMalloc(&sv->d_err, flag_bytes)) != cudaSuccess ||
      (e = cudaMemset(sv->d_err, 0, flag_bytes)) != cudaSuccess ||
      (e = cudaMallocHost(&sv->h_err, flag_bytes)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(sv->arena_base);
    cudaFree(sv->d_err);
    delete sv;
    return fail(nullptr, EGH_ENOMEM, std::string("error flags: ") + cudaGetErrorString(e));
  }
  std::memset(sv->h_err, 0, flag_bytes);
  sv->arena.reset((size_t)cfg->hbm_budget_bytes);
  sv->streams.resize(sv->nslots);
  sv->slot_busy.assign(sv->nslots, false);
  for (auto& s : sv->streams) cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  sv->worker = std::thread(worker_loop, sv);
  *out = sv;
  return EGH_OK;
}

egh_status egh_server_add_set(egh_server* sv, int32_t nrec, int32_t nfreq, const double* freq_hz,
                              double dt, int32_t nt_record, int32_t max_nt, const void* Q_host,
                              int32_t* set_id) {
  if (!sv || !freq_hz || !Q_host || !set_id) return fail(sv, EGH_EINVAL, "NULL argument");
  if (nrec < 1 || nfreq < 1 || nfreq > 64 || !(dt > 0) || nt_record < 1 || max_nt < 1)
    return fail(sv, EGH_EINVAL, "bad set dimensions");
  for (int k = 0; k < nfreq; ++k)
    if (!(freq_hz[k] > 0) || !(freq_hz[k] < 0.5 / dt))
      return fail(sv, EGH_EINVAL, "frequency outside (0, 1/(2 dt))");
  if (cudaSetDevice(sv->dev) != cudaSuccess) return fail(sv, EGH_ECUDA, "cudaSetDevice");
  HSet h;
  h.nrec = nrec;
  h.nf = nfreq;
  h.tw_len = max_nt;
  const std::vector<double> f(freq_hz, freq_hz + nfreq);
  const size_t qn = (size_t)nfreq * nrec * nrec;
  const std::vector<float2> tw = twiddle_table(f, dt, max_nt);
  const std::vector<float> w = synthesis_weights(f, dt, nt_record);
  int* status = nullptr;
  cudaStream_t st = sv->streams[0];
  double* d_cond = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_cond);
    cudaFree(h.kref);
    cudaFree(h.Ph);
    cudaFree(h.twt);
    cudaFree(h.tws);
    cudaFree(h.Wh);
    cudaFree(h.Qh);
    cudaFree(h.Lh);
    cudaFree(h.tw);
    cudaFree(h.w);
    cudaFree(status);
  };
  cudaError_t e = cudaSuccess;
  if (!e) e = cudaMalloc(&h.Qh, qn * sizeof(float2));
  if (!e) e = cudaMalloc(&h.Lh, qn * sizeof(float2));
  if (!e) e = cudaMalloc(&h.tw, tw.size() * sizeof(float2));
  if (!e) e = cudaMalloc(&h.w, w.size() * sizeof(float));
  if (!e) e = cudaMalloc(&status, nfreq * sizeof(int));
  if (!e) e = cudaMemcpy(h.Qh, Q_host, qn * sizeof(float2), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(h.Lh, Q_host, qn * sizeof(float2), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(h.tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (!e) {
    const std::vector<unsigned char> t = dft_twiddle_tiles(f, dt, max_nt);
    e = cudaMalloc(&h.twt, t.size());
    if (!e) e = cudaMemcpy(h.twt, t.data(), t.size(), cudaMemcpyHostToDevice);
  }
  if (!e) {
    const std::vector<unsigned char> u = synth_twiddle_tiles(f, dt, max_nt);
    e = cudaMalloc(&h.tws, u.size());
    if (!e) e = cudaMemcpy(h.tws, u.data(), u.size(), cudaMemcpyHostToDevice);
  }
  if (!e) e = cudaMemcpy(h.w, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (!e) e = launch_potrf(h.Lh, nrec, nfreq, status, st, prec_mixed(sv->prec) ? 1 : 0);
  std::vector<double> cond(2 * nfreq, 0.0);
  if (!e && prec_mixed(sv->prec)) {
    e = cudaMalloc(&h.Wh, qn * sizeof(float2));
    if (!e) e = launch_trtri(h.Lh, nrec, nfreq, h.Wh, st);
    if (!e) e = cudaMalloc(&h.Ph, qn * sizeof(float2));
    if (!e) e = launch_gram_inverse(h.Wh, nrec, nfreq, h.Ph, st);
    if (!e) e = cudaMalloc(&d_cond, 2 * nfreq * sizeof(double));
    if (!e) e = launch_fro2(h.Qh, nrec, nfreq, d_cond, st);
    if (!e) e = launch_inv_power(h.Wh, nrec, nfreq, d_cond + nfreq, st);
    if (!e) e = cudaMemcpyAsync(cond.data(), d_cond, 2 * nfreq * sizeof(double), cudaMemcpyDeviceToHost, st);
  }
  std::vector<int> stv(nfreq, 0);
  if (!e) e = cudaMemcpyAsync(stv.data(), status, nfreq * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (!e && prec_mixed(sv->prec)) {
    // selective refinement as for a context (the penalty of a set is not known: lambda_min comes
    // from the power estimate alone)
    std::vector<int> list;
    for (int k = 0; k < nfreq; ++k)
      if (cond_bound(cond[k], cond[nfreq + k], 0.0) > kRefineCond) list.push_back(k);
    h.nref = (int)list.size();
    if (!list.empty()) {
      e = cudaMalloc(&h.kref, list.size() * sizeof(int));
      if (!e) e = cudaMemcpy(h.kref, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
  }
  if (e) {
    cudaGetLastError();
    cleanup();
    return fail(sv, e == cudaErrorMemoryAllocation ? EGH_ENOMEM : EGH_ECUDA,
                std::string("egh_server_add_set: ") + cudaGetErrorString(e));
  }
  cudaFree(status);
  status = nullptr;
  cudaFree(d_cond);
  d_cond = nullptr;
  for (int k = 0; k < nfreq; ++k)
    if (stv[k]) {
      cleanup();
      return fail(sv, EGH_ENOTPD, "Hessian set not positive definite at frequency " + std::to_string(k));
    }
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->sets.push_back(h);
  *set_id = (int32_t)sv->sets.size() - 1;
  return EGH_OK;
}

egh_status egh_server_submit(egh_server* sv, int32_t set_id, const float* resid_host, int32_t ns,
                             int32_t nt_d, float* mult_host, int64_t* request_id) {
  if (!sv || !resid_host || !mult_host || !request_id) return fail(sv, EGH_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (!sv->worker_error.empty()) return fail(sv, EGH_ECUDA, sv->worker_error);
  if (set_id < 0 || set_id >= (int)sv->sets.size()) return fail(sv, EGH_EINVAL, "unknown set");
  const HSet& h = sv->sets[set_id];
  if (ns < 1 || nt_d < 1 || nt_d > h.tw_len)
    return fail(sv, EGH_EINVAL, "ns must be >= 1 and nt_d in 1..max_nt of the set");
  if ((long long)ns * h.nrec > 64LL * 65535) return fail(sv, EGH_EINVAL, "too many traces");
  Request* r = new (std::nothrow) Request();
  if (!r) return fail(sv, EGH_ENOMEM, "host allocation failed");
  r->set = set_id;
  r->ns = ns;
  r->nt_d = nt_d;
  r->resid = resid_host;
  r->mult = mult_host;
  r->bytes = trace_bytes(h, ns, nt_d);
  const size_t need = 2 * ((r->bytes + 255) / 256 * 256) + (d_bytes(sv, h, ns) + 255) / 256 * 256;
  if (need > sv->arena.total()) {
    delete r;
    ++sv->rejected;
    return fail(sv, EGH_ENOMEM, "request needs " + std::to_string(need) +
                                    " bytes, more than the server's HBM budget");
  }
  r->id = sv->next_id++;
  r->t_submit = now_s();
  if (sv->submitted == 0) sv->t_first = r->t_submit;
  ++sv->submitted;
  sv->reqs[r->id] = r;
  sv->queue.push_back(r);
  *request_id = r->id;
  sv->cv_work.notify_all();
  return EGH_OK;
}

egh_status egh_server_wait(egh_server* sv, int64_t request_id, double timeout_s, double* latency_s) {
  if (!sv) return fail(sv, EGH_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(request_id);
  if (it == sv->reqs.end()) return fail(sv, EGH_EINVAL, "unknown request");
  Request* r = it->second;
  const bool ok = sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                       [&] { return r->done || !sv->worker_error.empty(); });
  if (!r->done && sv->worker_error.empty() && !ok)
    return fail(sv, EGH_ETIMEOUT, "request not finished within the timeout (id kept)");
  // finished, failed, or never to run (the worker stopped): the id is released
  egh_status s = EGH_OK;
  std::string msg;
  if (r->done) {
    s = r->status;
    msg = r->msg;
    if (latency_s) *latency_s = r->t_done - r->t_submit;
  } else {
    s = EGH_ECUDA;
    msg = sv->worker_error;
    auto q = std::find(sv->queue.begin(), sv->queue.end(), r);
    if (q != sv->queue.end()) sv->queue.erase(q);
  }
  sv->reqs.erase(it);
  delete r;
  return s == EGH_OK ? EGH_OK : fail(sv, s, msg);
}

egh_status egh_server_drain(egh_server* sv, double timeout_s) {
  if (!sv) return fail(sv, EGH_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lk(sv->mu);
  const bool ok = sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
    return (sv->queue.empty() && sv->in_flight == 0) || !sv->worker_error.empty();
  });
  if (!sv->worker_error.empty()) return fail(sv, EGH_ECUDA, sv->worker_error);
  if (!ok) return fail(sv, EGH_ETIMEOUT, "requests still in flight after the timeout");
  // every batch has completed, so every batch's error flag has been read
  if (sv->device_timeouts) {
    const long long n = sv->device_timeouts;
    sv->device_timeouts = 0;
    return fail(sv, EGH_ETIMEOUT, std::to_string(n) + " batch(es) had a bounded device wait run out "
                                  "since the last drain (their requests returned EGH_ETIMEOUT)");
  }
  return EGH_OK;
}

egh_status egh_server_test_expire_wait(egh_server* sv, int32_t count) {
  if (!sv || count < 0) return fail(sv, EGH_EINVAL, "NULL server or negative count");
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->expire = count;
  return EGH_OK;
}

egh_status egh_server_get_stats(egh_server* sv, egh_server_stats* out) {
  if (!sv || !out) return fail(sv, EGH_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  egh_server_stats s{};
  s.submitted = sv->submitted;
  s.completed = sv->completed;
  s.rejected = sv->rejected;
  s.sources_done = sv->sources_done;
  s.batches = sv->batches;
  s.peak_in_flight = sv->peak_in_flight;
  s.peak_bytes_in_use = (int64_t)sv->arena.peak();
  s.span_s = sv->completed ? sv->t_last - sv->t_first : 0.0;
  if (!sv->latencies.empty()) {
    std::vector<double> v = sv->latencies;
    auto pct = [&](double q) {
      const size_t i = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
      std::nth_element(v.begin(), v.begin() + i, v.end());
      return v[i];
    };
    s.p50_s = pct(0.50);
    s.p99_s = pct(0.99);
    double m = 0;
    for (double x : sv->latencies) m += x;
    s.mean_s = m / (double)sv->latencies.size();
  }
  *out = s;
  return EGH_OK;
}

egh_status egh_server_hold(egh_server* sv, int32_t hold) {
  if (!sv) return fail(sv, EGH_EINVAL, "NULL server");
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->held = hold != 0;
  }
  sv->cv_work.notify_all();
  return EGH_OK;
}

egh_status egh_server_reset_stats(egh_server* sv) {
  if (!sv) return fail(sv, EGH_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->submitted = sv->completed = sv->rejected = sv->sources_done = sv->batches = 0;
  sv->latencies.clear();
  sv->peak_in_flight = sv->in_flight;
  sv->t_first = sv->t_last = 0;
  return EGH_OK;
}

const char* egh_server_last_error(const egh_server* sv) {
  return sv ? sv->err.c_str() : egh_last_error(nullptr);
}

void egh_server_destroy(egh_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  cudaSetDevice(sv->dev);
  for (auto& s : sv->streams) cudaStreamSynchronize(s);
  for (auto& s : sv->streams) cudaStreamDestroy(s);
  for (HSet& h : sv->sets) {
    cudaFree(h.kref);
    cudaFree(h.Ph);
    cudaFree(h.twt);
    cudaFree(h.tws);
    cudaFree(h.Wh);
    cudaFree(h.Qh);
    cudaFree(h.Lh);
    cudaFree(h.tw);
    cudaFree(h.w);
  }
  cudaFree(sv->arena_base);
  cudaFree(sv->d_err);
  cudaFreeHost(sv->h_err);
  for (auto& kv : sv->reqs) delete kv.second;
  delete sv;
}

}  // extern "C"
