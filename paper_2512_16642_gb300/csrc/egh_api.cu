// C ABI of the egh library: context, validation, device memory and the order of launches.
// Every numerical step runs in the kernels of fd.cu, gram.cu, chol.cu and deblur.cu; this file
// only validates, allocates, stages host buffers and sequences launches on the caller's stream.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "egh.h"
#include "egh_internal.cuh"

using namespace egh;

namespace {

// Eighth-order central second derivative (textbook coefficients).
const double kC8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
// Leapfrog stability bound on vmax dt sqrt(1/dx^2 + 1/dz^2) for that stencil:
// 2 / sqrt(205/72 + 2 (8/5 + 1/5 + 8/315 + 1/560)) = 0.784; kept with a small margin.
const double kCflMax = 0.78;

thread_local std::string g_create_error;
std::atomic<long long> g_launches{0};

enum State { ST_CREATED = 0, ST_GREEN = 1, ST_HESSIAN = 2, ST_FACTORED = 3 };

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

}  // namespace

namespace egh {
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
void set_context_free_error(const std::string& msg) { g_create_error = msg; }
}  // namespace egh

struct egh_ctx {
  int dev = 0;
  int nz = 0, nx = 0, ns = 0, nt = 0, nrec = 0, nf = 0;
  double dz = 0, dx = 0, R = 0, dt = 0;
  std::vector<int> rec_iz, rec_ix;
  std::vector<double> freqs;
  std::vector<float> wsyn;
  int B = 0, K = 0, splits = 0;
  int Bcap = 0;         // receivers the FD state slots hold (>= B)
  bool tune_B = false;  // B is timed on the first egh_green (8, 16 or 32 receivers)
  int fd_tz = 0;  // FD rows per warp of the per-step kernel (0 = library default)
  int fd_kernel = 2;  // 1: resident solver (fd_resident.cu), 2: one kernel per step (fd.cu)
  ResGeom rg{};       // resident solver: tile grid and pairs per block
  int res_sr = 0;     // resident solver: rows per z-march segment (0 = timed on first egh_green)
  float4* xbuf = nullptr;  // resident solver: halo exchange strips
  int* rflags = nullptr;   // resident solver: per-tile step counters + abort flag
  long long fd_steps = 0;  // last egh_green: FD steps computed
  int prec = EGH_PREC_FP32;
  int splits_tc = 0;  // grid-sum splits of the tensor-core Gram
  bool tune_splits = false;  // time half / once / twice the default splits on the first Gram
  Layout L{};
  Stencil S{};
  // device state
  float2 *coef = nullptr, *lev = nullptr;    // (c1, c3) per point; paired FD levels [3][B/2][F]
  __nv_bfloat16* snap = nullptr;             // [2][2K][Bp][G] hi/lo snapshots of the transform
  unsigned char* twt = nullptr;              // tensor-core twiddle tiles (64 levels each)
  unsigned char* twt_bl = nullptr;           // the same for the band-limited, decimated form
  size_t twt_bl_cap = 0;
  CUtensorMap tmap{};                        // TMA map of the snapshot ring (64-byte aligned type)
  int Bp = 0;                                // receivers per snapshot slot (B rounded up to even)
  float *gh = nullptr, *part = nullptr;
  __nv_bfloat16* ghb = nullptr;              // [nf][G/64][hi/lo][nrec x re/im][64] Gram operands
  CUtensorMap tmap_ghb{};                    // TMA map of ghb
  float2 *Qh = nullptr, *Lh = nullptr, *tw = nullptr;
  unsigned char* twt_deb = nullptr;  // the deblur transform's twiddle tiles (tw_len levels)
  unsigned char* tws_deb = nullptr;  // the synthesis twiddle tiles (tw_len samples)
  float2* Wh = nullptr;  // mixed precision: W = L^{-1} per frequency
  float2* Ph = nullptr;  // mixed precision: Q^{-1} = W^H W per frequency (solves as one product)
  double* fro2 = nullptr;  // mixed precision: ||Q_k||_F^2 of the last factorisation
  int* kref = nullptr;     // mixed precision: frequencies whose solves are refined (device list)
  int nref = 0;            // their number
  double refine_cond = kRefineCond;   // refinement threshold on the bound ||Q_k||_F / mu
  std::vector<double> cond_bound;     // the bound per frequency (last factorisation)
  std::vector<double> cond_host;      // its inputs: ||Q_k||_F^2, then 1 / lambda_min estimates
  std::vector<int> refined;           // 1 where the solves are refined
  int tw_len = 0;
  cudaStream_t side = nullptr;                 // the transform's stream inside egh_green (low priority)
  cudaStream_t fdst = nullptr;                 // the FD stream inside egh_green (high priority)
  // FD steps of a chunk as CUDA graphs, keyed by (first level mod 3, its offset in the chunk,
  // steps, ring slot of the chunk's level 0, pairs, rows per warp, levels per recorded level)
  std::map<std::tuple<int, int, int, int, int, int, int>, cudaGraphExec_t> fd_graphs;
  cudaEvent_t fd_done[2] = {}, dft_done[2] = {}, ev_side = nullptr;
  cudaEvent_t ev_tune[2] = {};                 // FD rows-per-warp timing
  cudaEvent_t ev_gram[2] = {};                 // the Gram kernel in the last egh_hessian
  // per-chunk start/end events of the FD steps and of the transform in the last egh_green
  std::vector<cudaEvent_t> ev_fd, ev_dft;
  long long fd_launches = 0, dft_launches = 0;
  float* w_dev = nullptr;
  int* rec_pts = nullptr;
  int* status = nullptr;
  double* dsum = nullptr;
  double* lmax = nullptr;
  float* vchk = nullptr;
  int* d_err = nullptr;  // set by bounded device waits that ran out
  int expire[3] = {0, 0, 0};  // test hook: launches (Green transform, resident FD, deblur
                              // transform) whose first block has one wait run out
  float* vel_stage = nullptr;
  float2* Dh = nullptr;
  size_t Dh_cap = 0;
  float2 *Dr = nullptr, *Rr = nullptr;  // refinement: right-hand sides kept, residuals
  size_t Dr_cap = 0, Rr_cap = 0;
  float *io_in = nullptr, *io_out = nullptr;
  size_t io_in_cap = 0, io_out_cap = 0;
  unsigned char* syn_ops = nullptr;  // the synthesis operand images
  size_t syn_ops_cap = 0;
  int state = ST_CREATED;
  double mu = 0;
  cudaEvent_t ev[8] = {};
  bool ev_rec[4] = {false, false, false, false};
  egh_stats st{};
  std::string err;
};


// Several contexts (survey patches of one model) whose Hessians are factored together.
struct egh_batch {
  std::vector<egh_ctx*> ctxs;
  int dev = 0, nmax = 0, count = 0, piv64 = 0, threads = 0;
  PotrfItem* items = nullptr;  // device list of every (context, frequency) matrix
  int* status = nullptr;       // device, one per item
  cudaStream_t cap = nullptr;  // capture stream
  cudaGraphExec_t graph = nullptr;
  int graph_launches = 0;      // kernels in one replay of the graph
  cudaEvent_t ev[2] = {};
  std::string err;
};

namespace {

egh_status fail(egh_ctx* c, egh_status s, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_create_error = msg;
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, EGH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

egh_status dalloc(egh_ctx* ctx, void** p, size_t bytes, const char* what) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    char buf[256];
    snprintf(buf, sizeof buf, "cudaMalloc(%s, %zu bytes): %s", what, bytes, cudaGetErrorString(e));
    return fail(ctx, e == cudaErrorMemoryAllocation ? EGH_ENOMEM : EGH_ECUDA, buf);
  }
  return EGH_OK;
}

// The device address of a page-locked host buffer mapped into the device's address space, or
// null (pageable memory, or no mapping).
void* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// 1 = device (or managed) memory, 0 = host memory (pinned or pageable).
int pointer_is_device(const void* p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? 1 : 0;
}

}  // namespace

namespace egh {
// exp(-i 2 pi f_k n dt) for n < len, phase reduced as 2 pi frac(f_k n dt) in double precision.
std::vector<float2> twiddle_table(const std::vector<double>& f, double dt, int len) {
  std::vector<float2> t((size_t)len * f.size());
  for (int n = 0; n < len; ++n)
    for (size_t k = 0; k < f.size(); ++k) {
      double ph = f[k] * (double)n * dt;
      ph -= std::floor(ph);
      const double a = 2.0 * M_PI * ph;
      t[(size_t)n * f.size() + k] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
  return t;
}

// Band-limited synthesis weights w_k = 2 df_k dt (df_k: half the distance between the
// neighbouring frequencies, the full gap at the ends, 1/(nt dt) for a single frequency).
std::vector<float> synthesis_weights(const std::vector<double>& f, double dt, int nt) {
  const int nf = (int)f.size();
  std::vector<double> df(nf);
  if (nf == 1) {
    df[0] = 1.0 / (nt * dt);
  } else {
    for (int k = 1; k < nf - 1; ++k) df[k] = 0.5 * (f[k + 1] - f[k - 1]);
    df[0] = f[1] - f[0];
    df[nf - 1] = f[nf - 1] - f[nf - 2];
  }
  std::vector<float> w(nf);
  for (int k = 0; k < nf; ++k) w[k] = (float)(2.0 * df[k] * dt);
  return w;
}
}  // namespace egh

namespace {

egh_status ensure_twiddles(egh_ctx* ctx, int len, cudaStream_t stream) {
  if (len <= ctx->tw_len) return EGH_OK;
  std::vector<float2> h = twiddle_table(ctx->freqs, ctx->dt, len);
  CK(cudaStreamSynchronize(stream));
  if (ctx->tw) CK(cudaFree(ctx->tw));
  if (ctx->twt_deb) CK(cudaFree(ctx->twt_deb));
  if (ctx->tws_deb) CK(cudaFree(ctx->tws_deb));
  ctx->tw = nullptr;
  ctx->twt_deb = nullptr;
  ctx->tws_deb = nullptr;
  ctx->tw_len = 0;
  egh_status s = dalloc(ctx, (void**)&ctx->tw, h.size() * sizeof(float2), "twiddles");
  if (s) return s;
  CK(cudaMemcpy(ctx->tw, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice));
  const std::vector<unsigned char> t = dft_twiddle_tiles(ctx->freqs, ctx->dt, len);
  if ((s = dalloc(ctx, (void**)&ctx->twt_deb, t.size(), "deblur twiddle tiles"))) return s;
  CK(cudaMemcpy(ctx->twt_deb, t.data(), t.size(), cudaMemcpyHostToDevice));
  const std::vector<unsigned char> u = synth_twiddle_tiles(ctx->freqs, ctx->dt, len);
  if ((s = dalloc(ctx, (void**)&ctx->tws_deb, u.size(), "synthesis twiddle tiles"))) return s;
  CK(cudaMemcpy(ctx->tws_deb, u.data(), u.size(), cudaMemcpyHostToDevice));
  ctx->tw_len = len;
  return EGH_OK;
}

egh_status ensure_buf(egh_ctx* ctx, void** p, size_t* cap, size_t bytes, cudaStream_t stream,
                      const char* what) {
  if (bytes <= *cap) return EGH_OK;
  CK(cudaStreamSynchronize(stream));
  if (*p) CK(cudaFree(*p));
  *p = nullptr;
  *cap = 0;
  egh_status s = dalloc(ctx, p, bytes, what);
  if (s) return s;
  *cap = bytes;
  return EGH_OK;
}

// Velocity validation (positive, finite, CFL) and coefficient build; returns the device pointer
// of the velocity actually used (the caller's, or the staging copy of a host array).
egh_status prepare_model(egh_ctx* ctx, const float* vel, cudaStream_t stream) {
  if (!vel) return fail(ctx, EGH_EINVAL, "velocity pointer is NULL");
  const long long n = (long long)ctx->nz * ctx->nx;
  const float* dv = vel;
  if (!pointer_is_device(vel)) {
    CK(cudaMemcpyAsync(ctx->vel_stage, vel, n * sizeof(float), cudaMemcpyHostToDevice, stream));
    dv = ctx->vel_stage;
  }
  CK(launch_check_velocity(dv, n, ctx->vchk, stream));
  float h[2];
  CK(cudaMemcpyAsync(h, ctx->vchk, sizeof h, cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  if (h[1] != 0.f) return fail(ctx, EGH_EINVAL, "velocity has non-positive or non-finite values");
  const double cfl = h[0] * ctx->dt * std::sqrt(1.0 / (ctx->dx * ctx->dx) + 1.0 / (ctx->dz * ctx->dz));
  if (cfl > kCflMax) {
    char buf[160];
    snprintf(buf, sizeof buf, "CFL number %.4f exceeds %.2f (vmax %.1f m/s)", cfl, kCflMax, h[0]);
    return fail(ctx, EGH_EINVAL, buf);
  }
  CK(launch_build_coef(dv, ctx->L, ctx->dz, ctx->dx, ctx->dt, ctx->R, ctx->vchk, ctx->coef, stream));
  return EGH_OK;
}

// FD state slot of level t: [3][B/2][F] float2.
float2* slot(egh_ctx* ctx, int t) {
  return ctx->lev + (long long)(t % 3) * ((ctx->Bcap + 1) / 2) * ctx->L.F;
}

// Snapshot output for ring slot j (0 .. 2K-1).
SnapOut snap_slot(egh_ctx* ctx, int j) {
  const long long per = (long long)ctx->Bp * ctx->L.G;
  return SnapOut{ctx->snap + (long long)j * per, 2LL * ctx->K * per, ctx->L.G};
}

// Zero both planes of ring slot j for the receivers of a batch.
cudaError_t zero_snap_slot(egh_ctx* ctx, int j, cudaStream_t st) {
  const SnapOut so = snap_slot(ctx, j);
  const size_t bytes = (size_t)ctx->Bp * ctx->L.G * sizeof(__nv_bfloat16);
  cudaError_t e = cudaMemsetAsync(so.lvl, 0, bytes, st);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(so.lvl + so.plane, 0, bytes, st);
}

void free_all(egh_ctx* c) {
  void* ptrs[] = {c->Ph, c->fro2, c->kref, c->xbuf, c->rflags, c->tws_deb, c->twt_deb, c->twt_bl, c->Wh, c->Dr, c->Rr, c->coef, c->lev, c->snap, c->twt, c->gh, c->ghb, c->part, c->Qh, c->Lh, c->tw, c->w_dev,
                  c->rec_pts, c->status, c->dsum, c->lmax, c->vchk, c->d_err, c->vel_stage, c->Dh,
                  c->io_in, c->io_out, c->syn_ops};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : {c->fd_done[0], c->fd_done[1], c->dft_done[0], c->dft_done[1], c->ev_side,
                        c->ev_tune[0], c->ev_tune[1], c->ev_gram[0], c->ev_gram[1]})
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_fd) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_dft) cudaEventDestroy(e);
  for (auto& kv : c->fd_graphs) cudaGraphExecDestroy(kv.second);
  c->fd_graphs.clear();
  if (c->side) cudaStreamDestroy(c->side);
  if (c->fdst) cudaStreamDestroy(c->fdst);
}


// The Green-stage buffers (snapshot ring, transforms, bf16 transforms) are the largest; egh_green
// allocates them on its first call and again after egh_release_green freed them.
egh_status ensure_green_buffers(egh_ctx* ctx, bool with_ring = true) {
  const Layout& L = ctx->L;
  const size_t snap_bytes = (size_t)2 * 2 * ctx->K * ctx->Bp * (size_t)L.G * sizeof(__nv_bfloat16);
  egh_status s;
  if (with_ring && !ctx->snap) {
    if ((s = dalloc(ctx, (void**)&ctx->snap, snap_bytes, "snapshot ring"))) return s;
    // padding points of every snapshot slot stay zero for the life of the buffer
    CK(cudaMemset(ctx->snap, 0, snap_bytes));
    CK(make_snap_tmap(&ctx->tmap, ctx->snap, L.G, ctx->Bp, 2 * ctx->K));
  }
  if (ctx->gh) return EGH_OK;
  if ((s = dalloc(ctx, (void**)&ctx->gh, (size_t)ctx->nrec * ctx->nf * 2 * (size_t)L.G * sizeof(float),
                  "green transforms")))
    return s;
  if (prec_mixed(ctx->prec) &&
      (s = dalloc(ctx, (void**)&ctx->ghb,
                  (size_t)ctx->nrec * ctx->nf * 4 * (size_t)L.G * sizeof(__nv_bfloat16),
                  "bf16 transforms")))
    return s;
  if (ctx->ghb) CK(make_ghb_tmap(&ctx->tmap_ghb, ctx->ghb, L.G, ctx->nf, ctx->nrec));
  return EGH_OK;
}

void release_green_buffers(egh_ctx* ctx) {
  cudaFree(ctx->snap);
  cudaFree(ctx->gh);
  cudaFree(ctx->ghb);
  ctx->snap = nullptr;
  ctx->gh = nullptr;
  ctx->ghb = nullptr;
  // graphs captured the ring slots' addresses
  for (auto& kv : ctx->fd_graphs) cudaGraphExecDestroy(kv.second);
  ctx->fd_graphs.clear();
}

// Snapshot output of level t in a chunk whose level t0 (a multiple of `decim`) sits in ring slot
// sbase: every decim-th level is recorded, the others write none.
SnapOut level_snap(egh_ctx* ctx, int t, int t0, int sbase, int decim) {
  if (t % decim) return SnapOut{nullptr, 0, 0};
  return snap_slot(ctx, sbase + (t - t0) / decim);
}

// FD steps t = ta .. t1-1 of a chunk whose level t0 sits in ring slot sbase, on the FD stream, as
// one CUDA graph (captured on first use, then replayed: the kernel nodes' arguments depend only
// on the key, since state slots follow t mod 3 and ring slots follow t - t0).
egh_status fd_chunk_steps(egh_ctx* ctx, int ta, int t0, int t1, int sbase, int np, int decim) {
  if (ta >= t1) return EGH_OK;
  const auto key = std::make_tuple(ta % 3, ta - t0, t1 - ta, sbase, np, ctx->fd_tz, decim);
  auto it = ctx->fd_graphs.find(key);
  if (it == ctx->fd_graphs.end()) {
    CK(cudaStreamBeginCapture(ctx->fdst, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int t = ta; t < t1 && e == cudaSuccess; ++t)
      e = launch_fd_step(slot(ctx, t - 1), slot(ctx, t - 2), slot(ctx, t), ctx->coef, ctx->L,
                         ctx->S, np, level_snap(ctx, t, t0, sbase, decim), ctx->fdst, ctx->fd_tz);
    count_launches(-(t1 - ta));  // counted again at each replay
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(ctx->fdst, &graph);
    if (e == cudaSuccess) e = e2;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess)
      return fail(ctx, EGH_ECUDA, std::string("FD chunk graph: ") + cudaGetErrorString(e));
    it = ctx->fd_graphs.emplace(key, exec).first;
  }
  CK(cudaGraphLaunch(it->second, ctx->fdst));
  count_launches(t1 - ta);
  return EGH_OK;
}

// Selective refinement of the mixed precisions, step 1 (queued on `stream` after the inverse
// factors): ||Q_k||_F^2 and the power estimate of 1 / lambda_min(Q_k), copied to the host buffer.
egh_status refine_plan(egh_ctx* ctx, cudaStream_t stream) {
  if (!ctx->Wh) return EGH_OK;
  CK(launch_fro2(ctx->Qh, ctx->nrec, ctx->nf, ctx->fro2, stream));
  CK(launch_inv_power(ctx->Wh, ctx->nrec, ctx->nf, ctx->fro2 + ctx->nf, stream));
  ctx->cond_host.assign(2 * ctx->nf, 0.0);
  CK(cudaMemcpyAsync(ctx->cond_host.data(), ctx->fro2, 2 * ctx->nf * sizeof(double),
                     cudaMemcpyDeviceToHost, stream));
  return EGH_OK;
}

// Step 2 (after the stream is synchronised): the solves of frequency k get one refinement step
// when its condition bound (||Q_k||_F over the smaller of mu and the power estimate of
// lambda_min) exceeds the threshold; the list goes to the device.
egh_status refine_list(egh_ctx* ctx) {
  if (!ctx->Wh) return EGH_OK;
  ctx->cond_bound.assign(ctx->nf, 0.0);
  ctx->refined.assign(ctx->nf, 0);
  std::vector<int> list;
  for (int k = 0; k < ctx->nf; ++k) {
    ctx->cond_bound[k] = cond_bound(ctx->cond_host[k], ctx->cond_host[ctx->nf + k], ctx->mu);
    if (ctx->cond_bound[k] > ctx->refine_cond) {
      list.push_back(k);
      ctx->refined[k] = 1;
    }
  }
  ctx->nref = (int)list.size();
  if (!list.empty())
    CK(cudaMemcpy(ctx->kref, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice));
  return EGH_OK;
}

}  // namespace

extern "C" {

int32_t egh_version(void) { return 10000; }

const char* egh_status_string(egh_status s) {
  switch (s) {
    case EGH_OK: return "EGH_OK";
    case EGH_EINVAL: return "EGH_EINVAL";
    case EGH_ENOMEM: return "EGH_ENOMEM";
    case EGH_ECUDA: return "EGH_ECUDA";
    case EGH_ENOTPD: return "EGH_ENOTPD";
    case EGH_ESTATE: return "EGH_ESTATE";
    case EGH_ETIMEOUT: return "EGH_ETIMEOUT";
  }
  return "EGH_UNKNOWN";
}

const char* egh_last_error(const egh_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

egh_status egh_create(const egh_config* cfg, egh_ctx** out) {
  egh_ctx* ctx = nullptr;
  if (!out) return fail(nullptr, EGH_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, EGH_EINVAL, "config is NULL");
  const egh_config& c = *cfg;
  for (int v : c.reserved)
    if (v != 0) return fail(nullptr, EGH_EINVAL, "reserved config fields must be zero");
  if (c.fd_kernel < 0 || c.fd_kernel > 2) return fail(nullptr, EGH_EINVAL, "fd_kernel must be 0, 1 or 2");
  if (c.nz < 1 || c.nx < 1) return fail(nullptr, EGH_EINVAL, "nz and nx must be >= 1");
  if (!(c.dz > 0) || !(c.dx > 0)) return fail(nullptr, EGH_EINVAL, "dz and dx must be > 0");
  if (c.nsponge < 0) return fail(nullptr, EGH_EINVAL, "nsponge must be >= 0");
  if (c.nsponge > 0 && !(c.sponge_R > 0 && c.sponge_R < 1))
    return fail(nullptr, EGH_EINVAL, "sponge_R must be in (0, 1)");
  if (!(c.dt > 0)) return fail(nullptr, EGH_EINVAL, "dt must be > 0");
  if (c.nt < 1) return fail(nullptr, EGH_EINVAL, "nt must be >= 1");
  if (c.nrec < 1 || !c.rec_iz || !c.rec_ix) return fail(nullptr, EGH_EINVAL, "need >= 1 receiver");
  if (c.nfreq < 1 || c.nfreq > 64 || !c.freq_hz)
    return fail(nullptr, EGH_EINVAL, "nfreq must be in 1..64");
  for (int r = 0; r < c.nrec; ++r)
    if (c.rec_iz[r] < 0 || c.rec_iz[r] >= c.nz || c.rec_ix[r] < 0 || c.rec_ix[r] >= c.nx)
      return fail(nullptr, EGH_EINVAL, "receiver outside the physical grid");
  for (int k = 0; k < c.nfreq; ++k)
    if (!(c.freq_hz[k] > 0) || !(c.freq_hz[k] < 0.5 / c.dt))
      return fail(nullptr, EGH_EINVAL, "frequency outside (0, 1/(2 dt))");
  if (c.fd_rows != 0 && c.fd_rows != 12 && c.fd_rows != 16 && c.fd_rows != 18 && c.fd_rows != 20 &&
      c.fd_rows != 24 && c.fd_rows != 32)
    return fail(nullptr, EGH_EINVAL, "fd_rows must be 0, 12, 16, 18, 20, 24 or 32");
  if (c.batch_receivers > 32) return fail(nullptr, EGH_EINVAL, "batch_receivers must be <= 32");
  if (c.precision != EGH_PREC_FP32 && !prec_mixed(c.precision))
    return fail(nullptr, EGH_EINVAL, "unknown precision");
  if (c.batch_receivers < 0 || c.gram_splits < 0)
    return fail(nullptr, EGH_EINVAL, "batch_receivers and gram_splits must be >= 0");
  if (c.dft_chunk != 0 && c.dft_chunk != 32 && c.dft_chunk != 64 && c.dft_chunk != 128 &&
      c.dft_chunk != 256 && c.dft_chunk != 512 && c.dft_chunk != 1024 &&
      c.dft_chunk != 2048)
    return fail(nullptr, EGH_EINVAL, "dft_chunk must be 0 or a power of two from 32 to 2048");

  ctx = new (std::nothrow) egh_ctx();
  if (!ctx) return fail(nullptr, EGH_ENOMEM, "host allocation failed");
  cudaGetDevice(&ctx->dev);
  ctx->nz = c.nz; ctx->nx = c.nx; ctx->ns = c.nsponge; ctx->nt = c.nt; ctx->nrec = c.nrec;
  ctx->nf = c.nfreq; ctx->dz = c.dz; ctx->dx = c.dx; ctx->R = c.nsponge > 0 ? c.sponge_R : 0.5;
  ctx->dt = c.dt;
  ctx->rec_iz.assign(c.rec_iz, c.rec_iz + c.nrec);
  ctx->rec_ix.assign(c.rec_ix, c.rec_ix + c.nrec);
  ctx->freqs.assign(c.freq_hz, c.freq_hz + c.nfreq);
  ctx->K = c.dft_chunk ? c.dft_chunk : 512;
  // a record shorter than the chunk is one chunk either way: keep the ring no longer than it
  while (ctx->K > 32 && ctx->K / 2 >= c.nt) ctx->K /= 2;
  ctx->fd_tz = c.fd_rows;

  Layout& L = ctx->L;
  L.nz = c.nz; L.nx = c.nx; L.ns = c.nsponge;
  L.NZ = c.nz + 2 * c.nsponge;
  L.NX = c.nx + 2 * c.nsponge;
  L.PX = (int)std::max<long long>(64, round_up(L.NX + 4, 64));
  L.F = (long long)(L.NZ + 2 * GUARD) * L.PX;
  L.org = (long long)GUARD * L.PX;
  L.G = round_up((long long)L.NZ * L.PX, 256);

  // FD solver: the per-step kernel, or on request the resident solver when the state of the
  // batch's pairs fits a block's shared memory
  {
    const int want = c.batch_receivers ? c.batch_receivers : 16;
    bool res = false;
    if (c.fd_kernel == 1) {
      res = fd_resident_plan(L, (want + 1) / 2, &ctx->rg) &&
            !(c.batch_receivers && (c.batch_receivers + 1) / 2 > ctx->rg.P);
      if (res) {
        const int np = (std::min(c.batch_receivers ? c.batch_receivers : 2 * ctx->rg.P, c.nrec) + 1) / 2;
        for (int sr : {6, 8, 11, 16})
          if (fd_resident_prepare(ctx->rg, sr, np) != cudaSuccess) res = false;
        cudaGetLastError();
      }
      if (!res && c.fd_kernel == 1) {
        delete ctx;
        return fail(nullptr, EGH_EINVAL,
                    "fd_kernel = 1: the batch's state does not fit a block's shared memory with one "
                    "block per SM resident (grid too large, or batch_receivers too many)");
      }
    }
    ctx->fd_kernel = res ? 1 : 2;
    if (res)
      ctx->B = c.batch_receivers ? std::min(c.batch_receivers, c.nrec) : std::min(c.nrec, 2 * ctx->rg.P);
    else
      ctx->B = c.batch_receivers ? std::min(c.batch_receivers, c.nrec) : std::min(c.nrec, 16);
    ctx->Bp = 2 * ((ctx->B + 1) / 2);
    // with the per-step kernel and no batch given, B is timed on the first egh_green among 8,
    // 16 and 32 receivers: the state slots hold the largest
    ctx->tune_B = !res && c.batch_receivers == 0 && c.nrec > 8;
    ctx->Bcap = ctx->tune_B ? std::min(c.nrec, 32) : ctx->B;
  }

  ctx->prec = c.precision;
  {
    const int ntile = gram_tiles(c.nrec);
    const long long pairs_nf = (long long)ntile * (ntile + 1) / 2 * c.nfreq;
    long long s = (3LL * 456 + pairs_nf - 1) / pairs_nf;
    s = std::max(1LL, std::min(s, L.G / 2048));
    ctx->splits = c.gram_splits ? c.gram_splits : (int)std::max(1LL, s);
    ctx->splits_tc = c.gram_splits ? c.gram_splits : gram_tc_splits(c.nrec, c.nfreq, L.G);
    ctx->tune_splits = c.gram_splits == 0;
  }

  for (int k = 0; k < 4; ++k) {
    ctx->S.cx[k] = (float)(kC8[k + 1] / (c.dx * c.dx));
    ctx->S.cz[k] = (float)(kC8[k + 1] / (c.dz * c.dz));
  }

  ctx->wsyn = synthesis_weights(ctx->freqs, c.dt, c.nt);

  egh_status s = EGH_OK;
  const size_t F = (size_t)L.F;
#define ALLOC(ptr, bytes, what)                                 \
  do {                                                          \
    s = dalloc(ctx, (void**)&(ptr), (bytes), what);             \
    if (s) {                                                    \
      g_create_error = ctx->err;                                \
      free_all(ctx);                                            \
      delete ctx;                                               \
      return s;                                                 \
    }                                                           \
  } while (0)
  ALLOC(ctx->coef, F * sizeof(float2), "coefficients");
  ALLOC(ctx->lev, (size_t)3 * ((ctx->Bcap + 1) / 2) * F * sizeof(float2), "FD state");
  if (ctx->fd_kernel == 1) {
    ALLOC(ctx->xbuf, fd_resident_xbuf_float4(ctx->rg) * sizeof(float4), "FD halo exchange");
    ALLOC(ctx->rflags, sizeof(int) * fd_resident_flags(ctx->rg), "FD step counters");
  }
  std::vector<unsigned char> twt = dft_twiddle_tiles(ctx->freqs, c.dt, c.nt);
  ALLOC(ctx->twt, twt.size(), "twiddle tiles");
  ALLOC(ctx->part,
        std::max(gram_workspace_floats(c.nrec, c.nfreq, ctx->splits),
                 gram_tc_workspace_floats(c.nrec, c.nfreq,
                                          ctx->tune_splits ? 2 * ctx->splits_tc : ctx->splits_tc)) *
            sizeof(float),
        "gram");
  ALLOC(ctx->Qh, (size_t)c.nfreq * c.nrec * c.nrec * sizeof(float2), "Qh");
  ALLOC(ctx->Lh, (size_t)c.nfreq * c.nrec * c.nrec * sizeof(float2), "Lh");
  if (prec_mixed(ctx->prec)) {
    ALLOC(ctx->Wh, (size_t)c.nfreq * c.nrec * c.nrec * sizeof(float2), "inverse factors");
    ALLOC(ctx->Ph, (size_t)c.nfreq * c.nrec * c.nrec * sizeof(float2), "inverse Hessians");
    ALLOC(ctx->fro2, (size_t)2 * c.nfreq * sizeof(double), "condition estimates");
    ALLOC(ctx->kref, (size_t)c.nfreq * sizeof(int), "refined frequencies");
  }
  ALLOC(ctx->w_dev, (size_t)c.nfreq * sizeof(float), "weights");
  ALLOC(ctx->rec_pts, (size_t)c.nrec * sizeof(int), "receivers");
  ALLOC(ctx->status, (size_t)c.nfreq * sizeof(int), "status");
  ALLOC(ctx->dsum, sizeof(double), "dsum");
  ALLOC(ctx->lmax, (size_t)c.nfreq * sizeof(double), "lmax");
  ALLOC(ctx->vchk, 2 * sizeof(float), "vchk");
  ALLOC(ctx->d_err, sizeof(int), "error flag");
  ALLOC(ctx->vel_stage, (size_t)c.nz * c.nx * sizeof(float), "velocity staging");
#undef ALLOC
  auto init = [&]() -> egh_status {
    CK(cudaMemset(ctx->coef, 0, F * sizeof(float2)));
    // guard rows and padding columns of every state slot, and the padding points of every
    // snapshot slot, stay zero for the life of the context
    CK(cudaMemset(ctx->lev, 0, (size_t)3 * ((ctx->Bcap + 1) / 2) * F * sizeof(float2)));

    CK(cudaMemcpy(ctx->twt, twt.data(), twt.size(), cudaMemcpyHostToDevice));
    CK(fd_prepare(c.nfreq));
    {
      // FD steps are a serial chain of short kernels: their stream gets the highest priority so
      // that their blocks are placed ahead of the transform's, which fills the rest of the GPU
      int least = 0, greatest = 0;
      CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
      CK(cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, least));
      CK(cudaStreamCreateWithPriority(&ctx->fdst, cudaStreamNonBlocking, greatest));
    }
    for (cudaEvent_t* e : {&ctx->fd_done[0], &ctx->fd_done[1], &ctx->dft_done[0], &ctx->dft_done[1],
                           &ctx->ev_side})
      CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    CK(cudaEventCreate(&ctx->ev_tune[0]));
    CK(cudaEventCreate(&ctx->ev_tune[1]));
    CK(cudaEventCreate(&ctx->ev_gram[0]));
    CK(cudaEventCreate(&ctx->ev_gram[1]));
    {
      // the smallest batch a timing of B can choose has the most chunks
      const int bmin = ctx->tune_B ? 8 : ctx->B;
      const long long nchunks = (long long)((c.nrec + bmin - 1) / bmin) * ((c.nt + ctx->K - 1) / ctx->K);
      ctx->ev_fd.assign(2 * nchunks, nullptr);
      ctx->ev_dft.assign(2 * nchunks, nullptr);
      for (cudaEvent_t& e : ctx->ev_fd) CK(cudaEventCreate(&e));
      for (cudaEvent_t& e : ctx->ev_dft) CK(cudaEventCreate(&e));
    }
    CK(cudaMemset(ctx->d_err, 0, sizeof(int)));
    std::vector<int> rp(c.nrec);
    for (int r = 0; r < c.nrec; ++r)
      rp[r] = (int)(L.org + (long long)(c.rec_iz[r] + c.nsponge) * L.PX + (c.rec_ix[r] + c.nsponge));
    CK(cudaMemcpy(ctx->rec_pts, rp.data(), rp.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->w_dev, ctx->wsyn.data(), ctx->wsyn.size() * sizeof(float),
                  cudaMemcpyHostToDevice));
    for (cudaEvent_t& e : ctx->ev) CK(cudaEventCreate(&e));
    egh_status s2 = ensure_twiddles(ctx, c.nt, 0);
    if (s2) return s2;
    CK(cudaDeviceSynchronize());
    return EGH_OK;
  };
  s = init();
  if (s) {
    g_create_error = ctx->err;
    free_all(ctx);
    delete ctx;
    return s;
  }
  ctx->st.nz_pad = L.NZ;
  ctx->st.nx_pad = L.NX;
  ctx->st.pitch = L.PX;
  ctx->st.batch_receivers = ctx->B;
  ctx->st.dft_chunk = ctx->K;
  ctx->st.gram_splits = prec_mixed(ctx->prec) ? ctx->splits_tc : ctx->splits;
  *out = ctx;
  return EGH_OK;
}

void egh_destroy(egh_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->dev);
  cudaDeviceSynchronize();
  free_all(ctx);
  delete ctx;
}

}  // extern "C"

namespace {

// The Green stage.  wav == nullptr: Dirac source (impulse at level 1), every level transformed
// with the table ctx->twt.  Otherwise the band-limited form: wavelet sample s_n is injected at
// the receiver into level n + 1, every decim-th level is recorded and transformed with `twt`
// (which folds in the factor decim and the division by the wavelet's spectrum).
// Receivers per batch, timed once per context before the ring (sized for the batch) exists: the
// FD step's time per receiver-step for 8, 16 and 32 receivers (each with its one-wave rows per
// warp; 24 steps on the state slots, which the run rewrites, best of three passes after a
// warm-up).  16 is kept unless another is 3% faster per receiver.  The transform's work per
// receiver does not depend on the batch, and it runs beside the FD steps for every choice.
egh_status tune_batch(egh_ctx* ctx, cudaStream_t stream) {
  const Layout& L = ctx->L;
  cudaStream_t fs = ctx->fdst;
  CK(cudaEventRecord(ctx->ev_tune[0], stream));  // after the coefficients
  CK(cudaStreamWaitEvent(fs, ctx->ev_tune[0], 0));
  const SnapOut none{nullptr, 0, 0};
  const int def_b = std::min(ctx->Bcap, 16);
  float best = 1e30f, def_per = 1e30f;
  int best_b = def_b;
  for (int b : {8, 16, 32}) {
    if (b > ctx->Bcap) continue;
    const int np = (b + 1) / 2, tz = fd_rows_one_wave(L, np);
    float tb = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      float ms = 0.f;
      CK(cudaEventRecord(ctx->ev_tune[0], fs));
      for (int t = 2; t < 26; ++t)
        CK(launch_fd_step(slot(ctx, t - 1), slot(ctx, t - 2), slot(ctx, t), ctx->coef, L, ctx->S,
                          np, none, fs, tz));
      CK(cudaEventRecord(ctx->ev_tune[1], fs));
      CK(cudaEventSynchronize(ctx->ev_tune[1]));
      CK(cudaEventElapsedTime(&ms, ctx->ev_tune[0], ctx->ev_tune[1]));
      if (rep > 0) tb = std::min(tb, ms);
    }
    const float per = tb / (float)b;
    if (per < best) {
      best = per;
      best_b = b;
    }
    if (b == def_b) def_per = per;
  }
  ctx->B = best < 0.97f * def_per ? best_b : def_b;
  ctx->Bp = 2 * ((ctx->B + 1) / 2);
  ctx->st.batch_receivers = ctx->B;
  ctx->tune_B = false;
  return EGH_OK;
}

egh_status green_run(egh_ctx* ctx, const float* vel, cudaStream_t stream, const float* wav, int nw,
                     int decim, const unsigned char* twt) {
  CK(cudaSetDevice(ctx->dev));
  ctx->state = ST_CREATED;
  egh_status s = prepare_model(ctx, vel, stream);
  if (s) return s;
  if (ctx->tune_B && (s = tune_batch(ctx, stream))) return s;
  s = ensure_green_buffers(ctx);
  if (s) return s;
  const Layout& L = ctx->L;
  const int K = ctx->K, B = ctx->B, nt = ctx->nt;
  CK(cudaEventRecord(ctx->ev[0], stream));
  // the FD and transform streams start after the coefficients
  CK(cudaEventRecord(ctx->ev_side, stream));
  CK(cudaStreamWaitEvent(ctx->side, ctx->ev_side, 0));
  CK(cudaStreamWaitEvent(ctx->fdst, ctx->ev_side, 0));
  cudaStream_t fs = ctx->fdst;
  const float src_scale = (float)(1.0 / (ctx->dx * ctx->dz));
  const long long per = (long long)ctx->Bp * L.G;  // snapshot ring: elements per slot
  // resident solver: levels ta .. t1-1 of a chunk whose level t0 sits in ring slot sbase
  auto resident = [&](int ta, int t0, int t1, int sbase, int np, int D, int sr, int expire) {
    return launch_fd_resident(ctx->rg, sr, ctx->lev, (ctx->Bcap + 1) / 2, L, ctx->coef, ctx->S, np, ta,
                              t1 - ta, t0, D, sbase, ctx->snap, per, 2LL * K * per, L.G, ctx->xbuf,
                              ctx->rflags, ctx->d_err, expire, fs);
  };
  if (ctx->fd_kernel == 1 && ctx->res_sr == 0) {
    // rows per z-march segment of the resident solver: time each choice on this grid (24 steps
    // of a full batch writing their snapshots, as the run does; the run rewrites every state and
    // ring slot it reads), best of three passes after a warm-up; the default is kept unless
    // another choice is 3% faster
    const int np = (std::min(B, ctx->nrec) + 1) / 2;
    const int def_sr = fd_resident_sr_default();
    float best = 1e30f, def_ms = 1e30f;
    int best_sr = def_sr;
    for (int sr : {6, 8, 11, 16}) {
      float sr_best = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {
        float ms = 0.f;
        CK(cudaEventRecord(ctx->ev_tune[0], fs));
        CK(resident(2, 0, 26, 0, np, 1, sr, 0));
        CK(cudaEventRecord(ctx->ev_tune[1], fs));
        CK(cudaEventSynchronize(ctx->ev_tune[1]));
        CK(cudaEventElapsedTime(&ms, ctx->ev_tune[0], ctx->ev_tune[1]));
        if (rep > 0) sr_best = std::min(sr_best, ms);
      }
      if (sr_best < best) {
        best = sr_best;
        best_sr = sr;
      }
      if (sr == def_sr) def_ms = sr_best;
    }
    int derr = 0;  // a wait that ran out in the timing pass
    CK(cudaMemcpy(&derr, ctx->d_err, sizeof derr, cudaMemcpyDeviceToHost));
    if (derr) {
      CK(cudaMemset(ctx->d_err, 0, sizeof(int)));
      return fail(ctx, EGH_ETIMEOUT, "a bounded wait for a neighbouring tile ran out in the FD solver");
    }
    ctx->res_sr = best < 0.97f * def_ms ? best_sr : def_sr;
  }
  if (ctx->fd_kernel == 2 && ctx->fd_tz == 0) {
    // Rows per warp of the FD step: time each choice on this grid (steps of a full batch that
    // write their snapshots, as the run does; the run below rewrites every state slot and ring
    // slot it reads), best of three passes of 24 steps per choice.
    const int np = (std::min(B, ctx->nrec) + 1) / 2;
    float best = 1e30f, def_ms = 1e30f;
    const int def_tz = fd_rows_one_wave(L, np);
    int best_tz = def_tz;
    for (int tz : {12, 16, 18, 20, 24, 32}) {
      float tz_best = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {  // the first pass warms up
        float ms = 0.f;
        CK(cudaEventRecord(ctx->ev_tune[0], fs));
        for (int t = 2; t < 26; ++t)
          CK(launch_fd_step(slot(ctx, t - 1), slot(ctx, t - 2), slot(ctx, t), ctx->coef, L, ctx->S,
                            np, snap_slot(ctx, t % (2 * K)), fs, tz));
        CK(cudaEventRecord(ctx->ev_tune[1], fs));
        CK(cudaEventSynchronize(ctx->ev_tune[1]));
        CK(cudaEventElapsedTime(&ms, ctx->ev_tune[0], ctx->ev_tune[1]));
        if (rep > 0) tz_best = std::min(tz_best, ms);
      }
      if (tz_best < best) {
        best = tz_best;
        best_tz = tz;
      }
      if (tz == def_tz) def_ms = tz_best;
    }
    // keep the one-wave choice unless another is clearly faster: the pass runs without the
    // transform beside it, and close calls there have gone either way in the full stage
    ctx->fd_tz = best < 0.97f * def_ms ? best_tz : def_tz;
  }
  const int D = decim;
  const int ntd = (nt + D - 1) / D;  // recorded levels 0, D, 2D, ... < nt
  const int nchunk = (ntd + K - 1) / K;
  long long fd_steps = 0, fd_kernel_launches = 0;
  long long g = 0;  // chunks so far over all batches: chunk g uses ring slots (g % 2) K ..
  for (int b0 = 0; b0 < ctx->nrec; b0 += B) {
    const int nb = std::min(B, ctx->nrec - b0);
    const int np = (nb + 1) / 2;
    for (int c = 0; c < nchunk; ++c, ++g) {
      // recorded levels m0 .. m1-1 of this chunk; time levels t0 .. t1-1
      const int m0 = c * K, m1 = std::min(ntd, m0 + K);
      const int t0 = m0 * D, t1 = std::min(nt, m1 * D);
      const int sbase = (int)(g & 1) * K;
      // this chunk's slots were read by the transform of chunk g - 2
      if (g >= 2) CK(cudaStreamWaitEvent(fs, ctx->dft_done[g & 1], 0));
      CK(cudaEventRecord(ctx->ev_fd[2 * g], fs));
      for (int t = t0; t < std::min(t1, 2); ++t) {
        // level 0 is zero; level 1 is the first source sample (the step from zero levels adds only
        // the source): the impulse, or s_0 of the wavelet
        const SnapOut so = level_snap(ctx, t, t0, sbase, D);
        CK(cudaMemsetAsync(slot(ctx, t), 0, (size_t)np * L.F * sizeof(float2), fs));
        if (so.lvl) CK(zero_snap_slot(ctx, sbase + (t - t0) / D, fs));
        if (t == 1)
          CK(launch_inject(slot(ctx, 1), L.F, ctx->rec_pts + b0, ctx->coef, nb, wav ? wav[0] : 1.0f,
                           src_scale, L.org, so, fs));
      }
      // levels that still take a wavelet sample: a step, then the injection, launched directly
      const int ta = std::max(t0, 2);
      const int tw = wav ? std::max(ta, std::min(t1, nw + 1)) : ta;
      for (int t = ta; t < tw; ++t) {
        const SnapOut so = level_snap(ctx, t, t0, sbase, D);
        CK(launch_fd_step(slot(ctx, t - 1), slot(ctx, t - 2), slot(ctx, t), ctx->coef, L, ctx->S, np,
                          so, fs, ctx->fd_tz));
        CK(launch_inject(slot(ctx, t), L.F, ctx->rec_pts + b0, ctx->coef, nb, wav[t - 1], src_scale,
                         L.org, so, fs));
      }
      if (ctx->fd_kernel == 1) {
        if (tw < t1) {
          const int expire = ctx->expire[1] > 0 ? 1 : 0;
          ctx->expire[1] -= expire;
          CK(resident(tw, t0, t1, sbase, np, D, ctx->res_sr, expire));
        }
      } else if ((s = fd_chunk_steps(ctx, tw, t0, t1, sbase, np, D))) {
        return s;
      }
      fd_steps += std::max(0, t1 - std::max(t0, 2));
      if (ctx->fd_kernel == 1 && tw < t1) ++fd_kernel_launches;
      CK(cudaEventRecord(ctx->ev_fd[2 * g + 1], fs));
      CK(cudaEventRecord(ctx->fd_done[g & 1], fs));
      CK(cudaStreamWaitEvent(ctx->side, ctx->fd_done[g & 1], 0));
      CK(cudaEventRecord(ctx->ev_dft[2 * g], ctx->side));
      const int expire = ctx->expire[0] > 0 ? 1 : 0;
      ctx->expire[0] -= expire;
      // Beside the next chunk's FD steps the transform takes one CTA per SM (sized to fit next
      // to two FD CTAs of a full batch); the record's last chunk runs alone and takes three.  With
      // more than 32 frequencies one CTA per SM no longer keeps pace with the FD steps (measured:
      // 40 frequencies on the salt grid, transform 5.9 s against FD steps 5.1 s per patch), so
      // there the transform takes one CTA per tile and fills the SMs between FD launches.
      const bool alone = b0 + B >= ctx->nrec && c == nchunk - 1;
      const bool slim = dft_ncomp(ctx->nf) <= 64 && ctx->fd_kernel != 1;
      const long long beside = fd_sm_smem((std::min(B, ctx->nrec) + 1) / 2, ctx->fd_tz);
      CK(launch_dft_tc(ctx->tmap, twt, ctx->nf, sbase, m1 - m0, m0, L, ctx->gh, ctx->ghb,
                       (m1 == ntd && ctx->ghb) ? 1 : 0, b0, nb, ctx->nrec, ctx->d_err, expire,
                       alone ? 3 : slim ? 1 : 0, (alone || !slim) ? 0 : beside, ctx->side));
      CK(cudaEventRecord(ctx->ev_dft[2 * g + 1], ctx->side));
      CK(cudaEventRecord(ctx->dft_done[g & 1], ctx->side));
    }
  }
  CK(cudaEventRecord(ctx->ev_side, ctx->side));
  CK(cudaStreamWaitEvent(stream, ctx->ev_side, 0));
  CK(cudaEventRecord(ctx->ev_tune[0], fs));
  CK(cudaStreamWaitEvent(stream, ctx->ev_tune[0], 0));
  CK(cudaEventRecord(ctx->ev[1], stream));
  ctx->ev_rec[0] = true;
  int derr = 0;
  CK(cudaMemcpyAsync(&derr, ctx->d_err, sizeof derr, cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  if (derr) {
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), stream));
    return fail(ctx, EGH_ETIMEOUT, "a bounded device wait ran out in the Green stage (staged snapshots "
                                   "in the transform, or a neighbouring tile in the FD solver)");
  }
  {
    // per-kernel device time of this call: FD steps (memsets, impulse and graph replay of each
    // chunk, on the FD stream) and the transform launches (on their own stream)
    double fd = 0, dft = 0;
    for (long long i = 0; i < g; ++i) {
      float a = 0, b = 0;
      CK(cudaEventElapsedTime(&a, ctx->ev_fd[2 * i], ctx->ev_fd[2 * i + 1]));
      CK(cudaEventElapsedTime(&b, ctx->ev_dft[2 * i], ctx->ev_dft[2 * i + 1]));
      fd += a;
      dft += b;
    }
    ctx->st.fd_ms = fd;
    ctx->st.dft_ms = dft;
    ctx->st.fd_launches = ctx->fd_kernel == 1 ? fd_kernel_launches
                                              : (long long)((ctx->nrec + B - 1) / B) * std::max(0, nt - 2);
    ctx->st.dft_launches = g;
    ctx->st.fd_steps = fd_steps;
    ctx->st.fd_kernel = ctx->fd_kernel;
    ctx->st.fd_tiles = ctx->fd_kernel == 1 ? ctx->rg.TR * ctx->rg.TC : 0;
  }
  ctx->st.pde_solves = ctx->nrec;
  ctx->st.point_steps = (long long)ctx->nrec * nt * L.NZ * L.NX;
  ctx->state = ST_GREEN;
  return EGH_OK;
}

}  // namespace

extern "C" {

egh_status egh_green(egh_ctx* ctx, const float* vel, void* stream_) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  return green_run(ctx, vel, (cudaStream_t)stream_, nullptr, 0, 1, ctx->twt);
}

egh_status egh_green_bandlimited(egh_ctx* ctx, const float* vel, const float* wavelet,
                                 int32_t nw, int32_t decim, void* stream_) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  if (!wavelet || nw < 1 || nw > ctx->nt)
    return fail(ctx, EGH_EINVAL, "need a wavelet of 1 .. nt samples");
  if (decim < 1 || decim > ctx->nt) return fail(ctx, EGH_EINVAL, "decim must be in 1 .. nt");
  for (int n = 0; n < nw; ++n)
    if (!std::isfinite(wavelet[n])) return fail(ctx, EGH_EINVAL, "wavelet samples must be finite");
  // spectral division and the decimation factor, folded into the twiddles:
  // g(w_k) = decim / S(w_k) * sum_m u_{m decim} exp(-i w_k m decim dt), S(w) = sum_n s_n e^{-i w n dt}
  std::vector<std::complex<double>> scale(ctx->nf);
  double smax = 0.0;
  for (int k = 0; k < ctx->nf; ++k) {
    std::complex<double> S(0.0, 0.0);
    for (int n = 0; n < nw; ++n) {
      double ph = ctx->freqs[k] * (double)n * ctx->dt;
      ph -= std::floor(ph);
      S += (double)wavelet[n] * std::polar(1.0, -2.0 * M_PI * ph);
    }
    scale[k] = S;
    smax = std::max(smax, std::abs(S));
  }
  for (int k = 0; k < ctx->nf; ++k) {
    if (!(std::abs(scale[k]) > 1e-6 * smax))
      return fail(ctx, EGH_EINVAL, "the wavelet's spectrum vanishes at frequency " + std::to_string(k));
    scale[k] = (double)decim / scale[k];
  }
  const int ntd = (ctx->nt + decim - 1) / decim;
  const std::vector<unsigned char> twt =
      dft_twiddle_tiles(ctx->freqs, ctx->dt * decim, ntd, &scale);
  CK(cudaSetDevice(ctx->dev));
  cudaStream_t stream = (cudaStream_t)stream_;
  if (twt.size() > ctx->twt_bl_cap) {
    CK(cudaStreamSynchronize(stream));
    CK(cudaDeviceSynchronize());
    cudaFree(ctx->twt_bl);
    ctx->twt_bl = nullptr;
    ctx->twt_bl_cap = 0;
    egh_status s = dalloc(ctx, (void**)&ctx->twt_bl, twt.size(), "band-limited twiddle tiles");
    if (s) return s;
    ctx->twt_bl_cap = twt.size();
  }
  // the previous Green stage may still read the table
  CK(cudaStreamSynchronize(ctx->side));
  CK(cudaMemcpy(ctx->twt_bl, twt.data(), twt.size(), cudaMemcpyHostToDevice));
  return green_run(ctx, vel, stream, wavelet, nw, decim, ctx->twt_bl);
}

egh_status egh_hessian(egh_ctx* ctx, egh_mu_mode mode, double mu_param, double* mu_out,
                       void* stream_) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  cudaStream_t stream = (cudaStream_t)stream_;
  CK(cudaSetDevice(ctx->dev));
  if (ctx->state < ST_GREEN || !ctx->gh)
    return fail(ctx, EGH_ESTATE, "egh_hessian needs egh_green first");
  if (!std::isfinite(mu_param) || mu_param < 0)
    return fail(ctx, EGH_EINVAL, "mu_param must be finite and >= 0");
  if (mode != EGH_MU_ABS && mode != EGH_MU_REL_MEANDIAG && mode != EGH_MU_REL_MAXEIG)
    return fail(ctx, EGH_EINVAL, "unknown mu mode");
  CK(cudaEventRecord(ctx->ev[2], stream));
  if (prec_mixed(ctx->prec) && ctx->tune_splits) {
    // grid-sum splits of the tensor-core Gram: time half, once and twice the default on this
    // problem (the result is discarded; the run below recomputes it) and keep the fastest
    const int base = ctx->splits_tc;
    const long long cap = ctx->L.G / (16LL * 64);
    float best = 1e30f;
    int best_s = base;
    for (int cand : {std::max(1, base / 2), base, 2 * base}) {
      if (cand > cap && cand != base) continue;
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {  // the first pass warms up
        CK(cudaEventRecord(ctx->ev_gram[0], stream));
        CK(launch_gram_tc(ctx->tmap_ghb, ctx->nrec, ctx->nf, ctx->L.G, cand, ctx->part,
                          ctx->d_err, stream));
        CK(launch_gram_tc_finish(ctx->part, ctx->nrec, ctx->nf, cand, ctx->Qh, stream));
        CK(cudaEventRecord(ctx->ev_gram[1], stream));
        CK(cudaEventSynchronize(ctx->ev_gram[1]));
        CK(cudaEventElapsedTime(&ms, ctx->ev_gram[0], ctx->ev_gram[1]));
      }
      if (ms < best) {
        best = ms;
        best_s = cand;
      }
    }
    ctx->splits_tc = best_s;
    ctx->st.gram_splits = best_s;
    ctx->tune_splits = false;
  }
  CK(cudaEventRecord(ctx->ev_gram[0], stream));
  if (prec_mixed(ctx->prec)) {
    CK(launch_gram_tc(ctx->tmap_ghb, ctx->nrec, ctx->nf, ctx->L.G, ctx->splits_tc, ctx->part,
                      ctx->d_err, stream));
    CK(cudaEventRecord(ctx->ev_gram[1], stream));
    CK(launch_gram_tc_finish(ctx->part, ctx->nrec, ctx->nf, ctx->splits_tc, ctx->Qh, stream));
  } else {
    CK(launch_gram_partial(ctx->gh, ctx->nrec, ctx->nf, ctx->L.G, ctx->splits, ctx->part, stream));
    CK(cudaEventRecord(ctx->ev_gram[1], stream));
    CK(launch_gram_finish(ctx->part, ctx->nrec, ctx->nf, ctx->splits, ctx->Qh, stream));
  }
  double mu = mu_param;
  if (mode == EGH_MU_REL_MEANDIAG) {
    CK(launch_diag_sum(ctx->Qh, ctx->nrec, ctx->nf, ctx->dsum, stream));
    double sum = 0;
    CK(cudaMemcpyAsync(&sum, ctx->dsum, sizeof sum, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    mu = mu_param * sum / ((double)ctx->nf * ctx->nrec);
  } else if (mode == EGH_MU_REL_MAXEIG) {
    CK(launch_lambda_max(ctx->Qh, ctx->nrec, ctx->nf, ctx->lmax, stream));
    std::vector<double> lm(ctx->nf);
    CK(cudaMemcpyAsync(lm.data(), ctx->lmax, lm.size() * sizeof(double), cudaMemcpyDeviceToHost,
                       stream));
    CK(cudaStreamSynchronize(stream));
    mu = mu_param * *std::max_element(lm.begin(), lm.end());
  }
  {
    int derr = 0;
    CK(cudaMemcpyAsync(&derr, ctx->d_err, sizeof derr, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (derr) {
      CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), stream));
      return fail(ctx, EGH_ETIMEOUT, "a bounded device wait ran out (in the Gram, or in an earlier "
                                     "deblur on device buffers)");
    }
  }
  if (!std::isfinite(mu)) return fail(ctx, EGH_EINVAL, "mu is not finite");
  {
    float gms = 0.f;
    CK(cudaEventElapsedTime(&gms, ctx->ev_gram[0], ctx->ev_gram[1]));
    ctx->st.gram_ms = gms;
  }
  CK(launch_add_mu_copy(ctx->Qh, ctx->Lh, ctx->nrec, ctx->nf, (float)mu, stream));
  CK(cudaEventRecord(ctx->ev[3], stream));
  ctx->ev_rec[1] = true;
  ctx->mu = mu;
  ctx->st.mu = mu;
  if (mu_out) *mu_out = mu;
  ctx->state = ST_HESSIAN;
  return EGH_OK;
}

egh_status egh_factor(egh_ctx* ctx, int32_t* bad_freq, void* stream_) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  cudaStream_t stream = (cudaStream_t)stream_;
  CK(cudaSetDevice(ctx->dev));
  if (bad_freq) *bad_freq = -1;
  if (ctx->state < ST_HESSIAN) return fail(ctx, EGH_ESTATE, "egh_factor needs egh_hessian first");
  const size_t bytes = (size_t)ctx->nf * ctx->nrec * ctx->nrec * sizeof(float2);
  CK(cudaEventRecord(ctx->ev[4], stream));
  CK(cudaMemcpyAsync(ctx->Lh, ctx->Qh, bytes, cudaMemcpyDeviceToDevice, stream));
  CK(launch_potrf(ctx->Lh, ctx->nrec, ctx->nf, ctx->status, stream,
                  prec_mixed(ctx->prec) ? 1 : 0));
  if (ctx->Wh) {
    CK(launch_trtri(ctx->Lh, ctx->nrec, ctx->nf, ctx->Wh, stream));
    CK(launch_gram_inverse(ctx->Wh, ctx->nrec, ctx->nf, ctx->Ph, stream));
  }
  egh_status rs = refine_plan(ctx, stream);  // queues its kernels; reads them after the sync
  if (rs) return rs;
  CK(cudaEventRecord(ctx->ev[5], stream));
  ctx->ev_rec[2] = true;
  std::vector<int> stv(ctx->nf);
  CK(cudaMemcpyAsync(stv.data(), ctx->status, stv.size() * sizeof(int), cudaMemcpyDeviceToHost,
                     stream));
  CK(cudaStreamSynchronize(stream));
  if ((rs = refine_list(ctx))) return rs;
  for (int k = 0; k < ctx->nf; ++k)
    if (stv[k]) {
      if (bad_freq) *bad_freq = k;
      ctx->state = ST_HESSIAN;
      char buf[128];
      snprintf(buf, sizeof buf, "Hessian at frequency %d not positive definite (pivot %d)", k,
               stv[k] - 1);
      return fail(ctx, EGH_ENOTPD, buf);
    }
  ctx->state = ST_FACTORED;
  return EGH_OK;
}

static egh_status deblur_common(egh_ctx* ctx, const float* resid, int32_t ns, int32_t nt_d,
                                float* mult, float2* X, cudaStream_t stream, bool diag = false) {
  if (diag && ctx->state < ST_HESSIAN)
    return fail(ctx, EGH_ESTATE, "egh_deblur_diag needs egh_hessian first");
  if (!diag && ctx->state < ST_FACTORED) return fail(ctx, EGH_ESTATE, "egh_deblur needs egh_factor first");
  if (ns < 0 || nt_d < 1) return fail(ctx, EGH_EINVAL, "ns must be >= 0 and nt_d >= 1");
  if (ns == 0) return EGH_OK;  // an empty gather: nothing is read or written (NULL allowed)
  if (!resid || (!mult && !X)) return fail(ctx, EGH_EINVAL, "NULL buffer");
  const long long ntr = (long long)ns * ctx->nrec;
  if ((ntr + 63) / 64 > 65535) return fail(ctx, EGH_EINVAL, "too many traces in one call");
  const bool dev_in = pointer_is_device(resid);
  const bool dev_out = X ? true : pointer_is_device(mult);
  if (X && !pointer_is_device(X)) return fail(ctx, EGH_EINVAL, "X must be device memory");
  if (!X && dev_in != dev_out)
    return fail(ctx, EGH_EINVAL, "resid and mult must both be host or both be device memory");
  egh_status s = ensure_twiddles(ctx, nt_d, stream);
  if (s) return s;
  const size_t nbytes = (size_t)ntr * nt_d * sizeof(float);
  // Page-locked host buffers are mapped into the device's address space: the forward transform
  // reads the residuals and the synthesis writes the multipliers through the mapping (over the
  // CPU-GPU link, no staging copy).  Pageable host memory is staged through device buffers.
  const float* din = resid;
  const float* in_map = dev_in ? nullptr : static_cast<const float*>(mapped_host(resid));
  if (in_map) {
    din = in_map;
  } else if (!dev_in) {
    if ((s = ensure_buf(ctx, (void**)&ctx->io_in, &ctx->io_in_cap, nbytes, stream, "resid staging")))
      return s;
    CK(cudaMemcpyAsync(ctx->io_in, resid, nbytes, cudaMemcpyHostToDevice, stream));
    din = ctx->io_in;
  }
  float2* D = X;
  if (!D) {
    if ((s = ensure_buf(ctx, (void**)&ctx->Dh, &ctx->Dh_cap,
                        (size_t)ctx->nf * ntr * sizeof(float2), stream, "deblur spectra")))
      return s;
    D = ctx->Dh;
  }
  float* dout = mult;
  float* out_map = (!X && !dev_out) ? static_cast<float*>(mapped_host(mult)) : nullptr;
  if (out_map) {
    dout = out_map;
  } else if (!X && !dev_out) {
    if ((s = ensure_buf(ctx, (void**)&ctx->io_out, &ctx->io_out_cap, nbytes, stream,
                        "mult staging")))
      return s;
    dout = ctx->io_out;
  }
  CK(cudaEventRecord(ctx->ev[6], stream));
  const int expire = ctx->expire[2] > 0 ? 1 : 0;
  ctx->expire[2] -= expire;
  CK(launch_trace_dft(din, (int)ntr, nt_d, ctx->nf, ctx->nrec, ns, 0, D, stream,
                      ctx->twt_deb, ctx->d_err, expire, in_map == nullptr));
  const size_t dbytes = (size_t)ctx->nf * ntr * sizeof(float2);
  const bool refine = !diag && prec_mixed(ctx->prec) && ctx->nref > 0;
  if (!diag && prec_mixed(ctx->prec) &&
      (s = ensure_buf(ctx, (void**)&ctx->Rr, &ctx->Rr_cap, dbytes, stream, "solve scratch")))
    return s;
  if (refine &&  // the refinement residual
      (s = ensure_buf(ctx, (void**)&ctx->Dr, &ctx->Dr_cap, dbytes, stream, "refinement residual")))
    return s;
  float2* Xs = D;  // the solutions the synthesis reads
  if (diag) {
    CK(launch_diag_solve(ctx->Qh, ctx->nrec, ctx->nf, D, ns, stream));
  } else if (prec_mixed(ctx->prec)) {
    // Y = Q^{-1} D, one product on the tensor cores; at the frequencies whose condition bound asks
    // for it, the residual R = D - Q Y to FP64-class accuracy and the correction Y += Q^{-1} R
    float2* Y = ctx->Rr;
    CK(launch_cmm_tc(ctx->Ph, ctx->nrec, ctx->nf, D, ns, Y, nullptr, ctx->d_err, stream));
    if (refine) {
      CK(launch_resid(ctx->Qh, ctx->nrec, ctx->nref, Y, D, ns, ctx->Dr,
                      ctx->prec == EGH_PREC_MIXED_FP64, stream, ctx->kref));
      CK(launch_cmm_tc(ctx->Ph, ctx->nrec, ctx->nref, ctx->Dr, ns, D, ctx->kref, ctx->d_err, stream));
      CK(launch_add_correction(Y, D, ntr, ctx->nref, stream, ctx->kref));
    }
    Xs = Y;
    if (X) CK(cudaMemcpyAsync(X, Y, dbytes, cudaMemcpyDeviceToDevice, stream));
  } else {
    CK(launch_trsm(ctx->Lh, ctx->nrec, ctx->nf, D, ns, stream));
  }
  if (!X) {
    const size_t ob = synth_operands_bytes(ctx->nf, ntr);
    if (!out_map &&
        (s = ensure_buf(ctx, (void**)&ctx->syn_ops, &ctx->syn_ops_cap, ob, stream, "synthesis operands")))
      return s;
    CK(launch_synth(Xs, ctx->nrec, ns, ns, 0, ctx->nf, ctx->w_dev, ctx->tw, nt_d, dout, stream,
                    ctx->tws_deb, ctx->d_err, out_map == nullptr, out_map ? nullptr : ctx->syn_ops,
                    out_map ? 0 : ctx->syn_ops_cap));
  }
  CK(cudaEventRecord(ctx->ev[7], stream));
  ctx->ev_rec[3] = true;
  ctx->st.deblur_sources = ns;
  if (!X && !dev_out) {
    if (!out_map) CK(cudaMemcpyAsync(mult, dout, nbytes, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
  } else if (!dev_in) {
    CK(cudaStreamSynchronize(stream));
  }
  if (!dev_in || (!X && !dev_out)) {  // synchronised: report a bounded wait that ran out
    int derr = 0;
    CK(cudaMemcpy(&derr, ctx->d_err, sizeof derr, cudaMemcpyDeviceToHost));
    if (derr) {
      CK(cudaMemset(ctx->d_err, 0, sizeof(int)));
      return fail(ctx, EGH_ETIMEOUT, "a bounded wait for staged twiddles ran out in the transform");
    }
  }
  return EGH_OK;
}

egh_status egh_deblur(egh_ctx* ctx, const float* resid, int32_t ns, int32_t nt_d, float* mult,
                      void* stream) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  CK(cudaSetDevice(ctx->dev));
  if (!mult && ns != 0) return fail(ctx, EGH_EINVAL, "mult is NULL");
  return deblur_common(ctx, resid, ns, nt_d, mult, nullptr, (cudaStream_t)stream);
}

egh_status egh_deblur_freq(egh_ctx* ctx, const float* resid, int32_t ns, int32_t nt_d, void* X,
                           void* stream) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  CK(cudaSetDevice(ctx->dev));
  if (!X && ns != 0) return fail(ctx, EGH_EINVAL, "X is NULL");
  return deblur_common(ctx, resid, ns, nt_d, nullptr, (float2*)X, (cudaStream_t)stream);
}

egh_status egh_deblur_diag(egh_ctx* ctx, const float* resid, int32_t ns, int32_t nt_d, float* mult,
                           void* stream) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  CK(cudaSetDevice(ctx->dev));
  if (!mult && ns != 0) return fail(ctx, EGH_EINVAL, "mult is NULL");
  return deblur_common(ctx, resid, ns, nt_d, mult, nullptr, (cudaStream_t)stream, true);
}

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA
// 2014) used as a counter-based generator: output i = mix(seed + (i + 1) * golden gamma).
static uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

egh_status egh_sample_receivers(int32_t nrec, int32_t nsub, uint64_t seed, uint64_t iteration,
                                int32_t* out) {
  if (!out) return fail(nullptr, EGH_EINVAL, "out is NULL");
  if (nrec < 1 || nsub < 1 || nsub > nrec)
    return fail(nullptr, EGH_EINVAL, "need 1 <= nsub <= nrec");
  for (int32_t j = 0; j < nsub; ++j) {
    const int64_t lo = (int64_t)j * nrec / nsub, hi = (int64_t)(j + 1) * nrec / nsub;
    const uint64_t x = splitmix64_at(seed, iteration * (uint64_t)nsub + (uint64_t)j);
    const uint64_t pick = (uint64_t)(((unsigned __int128)x * (uint64_t)(hi - lo)) >> 64);
    out[j] = (int32_t)(lo + (int64_t)pick);
  }
  return EGH_OK;
}

egh_status egh_forward(egh_ctx* ctx, const float* vel, int32_t nsrc, const int32_t* src_iz,
                       const int32_t* src_ix, const float* wavelet, float* data, void* stream_) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  cudaStream_t stream = (cudaStream_t)stream_;
  CK(cudaSetDevice(ctx->dev));
  if (nsrc < 1 || !src_iz || !src_ix || !wavelet || !data)
    return fail(ctx, EGH_EINVAL, "bad forward-modelling arguments");
  for (int s = 0; s < nsrc; ++s)
    if (src_iz[s] < 0 || src_iz[s] >= ctx->nz || src_ix[s] < 0 || src_ix[s] >= ctx->nx)
      return fail(ctx, EGH_EINVAL, "source outside the physical grid");
  const int prev_state = ctx->state;
  egh_status s = prepare_model(ctx, vel, stream);
  ctx->state = prev_state;
  if (s) return s;
  const Layout& L = ctx->L;
  const int B = ctx->B, nt = ctx->nt, nrec = ctx->nrec;
  std::vector<int> sp(nsrc);
  for (int i = 0; i < nsrc; ++i)
    sp[i] = (int)(L.org + (long long)(src_iz[i] + L.ns) * L.PX + (src_ix[i] + L.ns));
  int* d_sp = nullptr;
  if ((s = dalloc(ctx, (void**)&d_sp, sp.size() * sizeof(int), "source points"))) return s;
  struct Guard {
    int* p;
    ~Guard() { cudaFree(p); }
  } guard{d_sp};
  CK(cudaMemcpyAsync(d_sp, sp.data(), sp.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
  const bool dev_out = pointer_is_device(data);
  const size_t nbytes = (size_t)nsrc * nrec * nt * sizeof(float);
  float* dout = data;
  if (!dev_out) {
    if ((s = ensure_buf(ctx, (void**)&ctx->io_out, &ctx->io_out_cap, nbytes, stream, "traces")))
      return s;
    dout = ctx->io_out;
  }
  const float scale = (float)(1.0 / (ctx->dx * ctx->dz));
  const SnapOut none{nullptr, 0, 0};
  for (int b0 = 0; b0 < nsrc; b0 += B) {
    const int nb = std::min(B, nsrc - b0);
    const int np = (nb + 1) / 2;
    float* tr = dout + (size_t)b0 * nrec * nt;
    CK(cudaMemsetAsync(slot(ctx, 0), 0, (size_t)np * L.F * sizeof(float2), stream));
    CK(cudaMemsetAsync(slot(ctx, 1), 0, (size_t)np * L.F * sizeof(float2), stream));
    CK(launch_record(slot(ctx, 0), L.F, ctx->rec_pts, nrec, nb, tr, nt, 0, stream));
    for (int n = 0; n + 1 < nt; ++n) {
      if (n > 0)
        CK(launch_fd_step(slot(ctx, n), slot(ctx, n - 1), slot(ctx, n + 1), ctx->coef, L, ctx->S,
                          np, none, stream, ctx->fd_tz));
      if (wavelet[n] != 0.f)
        CK(launch_inject(slot(ctx, n + 1), L.F, d_sp + b0, ctx->coef, nb, wavelet[n], scale, L.org,
                         none, stream));
      CK(launch_record(slot(ctx, n + 1), L.F, ctx->rec_pts, nrec, nb, tr, nt, n + 1, stream));
    }
  }
  if (!dev_out) CK(cudaMemcpyAsync(data, dout, nbytes, cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  return EGH_OK;
}

egh_status egh_get_green(egh_ctx* ctx, int32_t r0, int32_t nr, void* host_out) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  CK(cudaSetDevice(ctx->dev));
  if (ctx->state < ST_GREEN || !ctx->gh) return fail(ctx, EGH_ESTATE, "no Green functions yet");
  if (r0 < 0 || nr < 0 || r0 + nr > ctx->nrec || !host_out)
    return fail(ctx, EGH_EINVAL, "bad receiver range");
  CK(cudaDeviceSynchronize());
  const Layout& L = ctx->L;
  const size_t per = (size_t)ctx->nf * 2 * L.G;
  std::vector<float> h(per);
  float* out = (float*)host_out;
  for (int r = 0; r < nr; ++r) {
    CK(cudaMemcpy(h.data(), ctx->gh + (size_t)(r0 + r) * per, per * sizeof(float),
                  cudaMemcpyDeviceToHost));
    for (int k = 0; k < ctx->nf; ++k) {
      const float* re = h.data() + (size_t)k * 2 * L.G;
      const float* im = re + L.G;
      float* o = out + (((size_t)r * ctx->nf + k) * L.NZ * L.NX) * 2;
      for (int z = 0; z < L.NZ; ++z)
        for (int x = 0; x < L.NX; ++x) {
          const size_t p = (size_t)z * L.PX + x;
          o[2 * ((size_t)z * L.NX + x)] = re[p];
          o[2 * ((size_t)z * L.NX + x) + 1] = im[p];
        }
    }
  }
  return EGH_OK;
}

egh_status egh_get_hessian(egh_ctx* ctx, int32_t factored, void* host_out) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  CK(cudaSetDevice(ctx->dev));
  if (!host_out) return fail(ctx, EGH_EINVAL, "host_out is NULL");
  if (ctx->state < (factored ? ST_FACTORED : ST_HESSIAN))
    return fail(ctx, EGH_ESTATE, factored ? "no factors yet" : "no Hessian yet");
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(host_out, factored ? ctx->Lh : ctx->Qh,
                (size_t)ctx->nf * ctx->nrec * ctx->nrec * sizeof(float2), cudaMemcpyDeviceToHost));
  return EGH_OK;
}

egh_status egh_get_stats(egh_ctx* ctx, egh_stats* out) {
  if (!ctx || !out) return fail(ctx, EGH_EINVAL, "NULL argument");
  CK(cudaSetDevice(ctx->dev));
  double* ms[4] = {&ctx->st.green_ms, &ctx->st.hessian_ms, &ctx->st.factor_ms, &ctx->st.deblur_ms};
  for (int i = 0; i < 4; ++i)
    if (ctx->ev_rec[i]) {
      CK(cudaEventSynchronize(ctx->ev[2 * i + 1]));
      float t = 0;
      CK(cudaEventElapsedTime(&t, ctx->ev[2 * i], ctx->ev[2 * i + 1]));
      *ms[i] = t;
    }
  ctx->st.kernel_launches = launches_so_far();
  ctx->st.fd_rows = ctx->fd_kernel == 1 ? ctx->res_sr : ctx->fd_tz;
  ctx->st.fd_kernel = ctx->fd_kernel;
  ctx->st.fd_tiles = ctx->fd_kernel == 1 ? ctx->rg.TR * ctx->rg.TC : 0;
  *out = ctx->st;
  return EGH_OK;
}

egh_status egh_export_green(egh_ctx* ctx, int32_t k0, int32_t nk, float* d_out, void* stream_) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  CK(cudaSetDevice(ctx->dev));
  if (ctx->state < ST_GREEN || !ctx->gh) return fail(ctx, EGH_ESTATE, "egh_export_green needs egh_green first");
  if (k0 < 0 || nk < 0 || k0 + nk > ctx->nf) return fail(ctx, EGH_EINVAL, "frequency range outside 0..nfreq");
  if (nk == 0) return EGH_OK;
  if (!d_out || !pointer_is_device(d_out)) return fail(ctx, EGH_EINVAL, "d_out must be device memory");
  const size_t plane = 2 * (size_t)ctx->L.G * sizeof(float);  // one frequency of one receiver
  CK(cudaMemcpy2DAsync(d_out, nk * plane, ctx->gh + (size_t)k0 * 2 * ctx->L.G, ctx->nf * plane,
                       nk * plane, ctx->nrec, cudaMemcpyDeviceToDevice, (cudaStream_t)stream_));
  return EGH_OK;
}

egh_status egh_import_green(egh_ctx* ctx, const float* d_in, void* stream_) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  CK(cudaSetDevice(ctx->dev));
  if (!d_in || !pointer_is_device(d_in)) return fail(ctx, EGH_EINVAL, "d_in must be device memory");
  cudaStream_t stream = (cudaStream_t)stream_;
  ctx->state = ST_CREATED;
  egh_status s = ensure_green_buffers(ctx, false);  // no snapshot ring: no solve runs here
  if (s) return s;
  const size_t n = (size_t)ctx->nrec * ctx->nf * 2 * ctx->L.G;
  CK(cudaMemcpyAsync(ctx->gh, d_in, n * sizeof(float), cudaMemcpyDeviceToDevice, stream));
  if (ctx->ghb) CK(launch_gh_to_ghb(ctx->gh, ctx->nrec, ctx->nf, ctx->L.G, ctx->ghb, stream));
  CK(cudaStreamSynchronize(stream));
  ctx->st.pde_solves = 0;
  ctx->st.point_steps = 0;
  ctx->state = ST_GREEN;
  return EGH_OK;
}

egh_status egh_diag_sum(egh_ctx* ctx, double* out) {
  if (!ctx || !out) return fail(ctx, EGH_EINVAL, "NULL argument");
  CK(cudaSetDevice(ctx->dev));
  if (ctx->state < ST_HESSIAN) return fail(ctx, EGH_ESTATE, "egh_diag_sum needs egh_hessian first");
  CK(launch_diag_sum(ctx->Qh, ctx->nrec, ctx->nf, ctx->dsum, 0));
  CK(cudaMemcpy(out, ctx->dsum, sizeof(double), cudaMemcpyDeviceToHost));
  return EGH_OK;
}

egh_status egh_set_mu(egh_ctx* ctx, double mu, void* stream_) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  CK(cudaSetDevice(ctx->dev));
  if (ctx->state < ST_HESSIAN) return fail(ctx, EGH_ESTATE, "egh_set_mu needs egh_hessian first");
  if (!std::isfinite(mu) || mu < 0) return fail(ctx, EGH_EINVAL, "mu must be finite and >= 0");
  cudaStream_t stream = (cudaStream_t)stream_;
  CK(launch_add_mu_copy_delta(ctx->Qh, ctx->Lh, ctx->nrec, ctx->nf, ctx->mu, mu, stream));
  CK(cudaStreamSynchronize(stream));
  ctx->mu = mu;
  ctx->st.mu = mu;
  ctx->state = ST_HESSIAN;
  return EGH_OK;
}

egh_status egh_set_synthesis_frequencies(egh_ctx* ctx, const double* all_freq_hz, int32_t nall,
                                         int32_t k0) {
  if (!ctx || !all_freq_hz) return fail(ctx, EGH_EINVAL, "NULL argument");
  CK(cudaSetDevice(ctx->dev));
  if (nall < ctx->nf || k0 < 0 || k0 + ctx->nf > nall)
    return fail(ctx, EGH_EINVAL, "the context's frequencies must be entries k0.. of the full list");
  for (int k = 0; k < ctx->nf; ++k)
    if (all_freq_hz[k0 + k] != ctx->freqs[k])
      return fail(ctx, EGH_EINVAL, "the full list's entries k0.. differ from the context's frequencies");
  const std::vector<double> f(all_freq_hz, all_freq_hz + nall);
  const std::vector<float> w = synthesis_weights(f, ctx->dt, ctx->nt);
  ctx->wsyn.assign(w.begin() + k0, w.begin() + k0 + ctx->nf);
  CK(cudaMemcpy(ctx->w_dev, ctx->wsyn.data(), ctx->wsyn.size() * sizeof(float), cudaMemcpyHostToDevice));
  return EGH_OK;
}

egh_status egh_set_refinement(egh_ctx* ctx, double threshold) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  if (!(threshold >= 0)) return fail(ctx, EGH_EINVAL, "threshold must be >= 0 (inf: never refine)");
  ctx->refine_cond = threshold;
  return EGH_OK;
}

egh_status egh_get_refinement(egh_ctx* ctx, double* cond_bound, int32_t* refined) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  if (!prec_mixed(ctx->prec)) return fail(ctx, EGH_EINVAL, "only the mixed precisions refine");
  if (ctx->state < ST_FACTORED || ctx->cond_bound.empty())
    return fail(ctx, EGH_ESTATE, "egh_get_refinement needs egh_factor first");
  for (int k = 0; k < ctx->nf; ++k) {
    if (cond_bound) cond_bound[k] = ctx->cond_bound[k];
    if (refined) refined[k] = ctx->refined[k];
  }
  return EGH_OK;
}

egh_status egh_test_expire_wait(egh_ctx* ctx, int32_t kind, int32_t count) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  if (count < 0 || kind < 0 || kind > 2) return fail(ctx, EGH_EINVAL, "kind must be 0..2, count >= 0");
  if (kind == 1 && ctx->fd_kernel != 1)
    return fail(ctx, EGH_EINVAL, "this context does not use the resident FD solver");
  ctx->expire[kind] = count;
  return EGH_OK;
}

egh_status egh_release_green(egh_ctx* ctx) {
  if (!ctx) return fail(nullptr, EGH_EINVAL, "ctx is NULL");
  CK(cudaSetDevice(ctx->dev));
  CK(cudaDeviceSynchronize());
  release_green_buffers(ctx);
  return EGH_OK;
}

static egh_status bfail(egh_batch* b, egh_status s, const std::string& msg) {
  if (b)
    b->err = msg;
  else
    set_context_free_error(msg);
  return s;
}

#define BCK(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return bfail(b, EGH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

void egh_batch_destroy(egh_batch* b) {
  if (!b) return;
  cudaSetDevice(b->dev);
  cudaDeviceSynchronize();
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  cudaFree(b->items);
  cudaFree(b->status);
  delete b;
}

egh_status egh_batch_create(egh_ctx* const* ctxs, int32_t n, egh_batch** out) {
  if (!out || !ctxs || n < 1) return bfail(nullptr, EGH_EINVAL, "need >= 1 context");
  *out = nullptr;
  egh_batch* b = new (std::nothrow) egh_batch();
  if (!b) return bfail(nullptr, EGH_ENOMEM, "host allocation failed");
  std::vector<PotrfItem> items;
  for (int i = 0; i < n; ++i) {
    egh_ctx* c = ctxs[i];
    if (!c) {
      delete b;
      return bfail(nullptr, EGH_EINVAL, "NULL context in the batch");
    }
    if (i > 0 && (c->dev != ctxs[0]->dev || c->prec != ctxs[0]->prec)) {
      delete b;
      return bfail(nullptr, EGH_EINVAL, "batched contexts must share device and precision");
    }
    b->ctxs.push_back(c);
    b->nmax = std::max(b->nmax, c->nrec);
  }
  b->dev = ctxs[0]->dev;
  b->piv64 = prec_mixed(ctxs[0]->prec) ? 1 : 0;
  cudaSetDevice(b->dev);
  int off = 0;
  for (egh_ctx* c : b->ctxs) off += c->nf;
  b->count = off;
  auto setup = [&]() -> egh_status {
    BCK(cudaMalloc(&b->status, sizeof(int) * b->count));
    BCK(cudaMalloc(&b->items, sizeof(PotrfItem) * b->count));
    int o = 0;
    for (egh_ctx* c : b->ctxs)
      for (int k = 0; k < c->nf; ++k, ++o)
        items.push_back(PotrfItem{c->Lh + (size_t)k * c->nrec * c->nrec, c->nrec, b->status + o});
    BCK(cudaMemcpy(b->items, items.data(), sizeof(PotrfItem) * items.size(), cudaMemcpyHostToDevice));
    BCK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    BCK(cudaEventCreate(&b->ev[0]));
    BCK(cudaEventCreate(&b->ev[1]));
    BCK(potrf_many_prepare(b->nmax));
    return EGH_OK;
  };
  egh_status s = setup();
  if (s) {
    const std::string m = b->err;
    egh_batch_destroy(b);
    return bfail(nullptr, s, m);
  }
  *out = b;
  return EGH_OK;
}

// Q -> L copies of every context and one persistent factorisation launch, on `st`.
static cudaError_t batch_enqueue(egh_batch* b, int threads, cudaStream_t st) {
  cudaError_t e;
  for (egh_ctx* c : b->ctxs)
    if ((e = cudaMemcpyAsync(c->Lh, c->Qh, (size_t)c->nf * c->nrec * c->nrec * sizeof(float2),
                             cudaMemcpyDeviceToDevice, st)))
      return e;
  if ((e = launch_potrf_many(b->items, b->count, b->nmax, std::min(b->count, 2 * 152), threads,
                             b->piv64, st)))
    return e;
  for (egh_ctx* c : b->ctxs) {
    if (c->Wh && (e = launch_trtri(c->Lh, c->nrec, c->nf, c->Wh, st))) return e;
    if (c->Ph && (e = launch_gram_inverse(c->Wh, c->nrec, c->nf, c->Ph, st))) return e;
  }
  return cudaSuccess;
}

egh_status egh_batch_factor(egh_batch* b, int32_t* bad_ctx, int32_t* bad_freq, void* stream_) {
  if (!b) return bfail(nullptr, EGH_EINVAL, "batch is NULL");
  cudaStream_t stream = (cudaStream_t)stream_;
  if (bad_ctx) *bad_ctx = -1;
  if (bad_freq) *bad_freq = -1;
  BCK(cudaSetDevice(b->dev));
  for (egh_ctx* c : b->ctxs)
    if (c->state < ST_HESSIAN) return bfail(b, EGH_ESTATE, "every context needs egh_hessian first");
  if (!b->graph) {
    // launch shape: time each block size on these matrices and keep the fastest; then capture
    // the copies and the launch once as a CUDA graph
    float best = 1e30f;
    const long long l0 = launches_so_far();
    for (int th : {256, 512, 1024}) {
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        BCK(cudaEventRecord(b->ev[0], stream));
        BCK(batch_enqueue(b, th, stream));
        BCK(cudaEventRecord(b->ev[1], stream));
        BCK(cudaEventSynchronize(b->ev[1]));
        BCK(cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
      }
      if (ms < best) {
        best = ms;
        b->threads = th;
      }
    }
    count_launches(-(int)(launches_so_far() - l0));  // tuning launches are not part of the factorisation
    const long long l1 = launches_so_far();
    BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = batch_enqueue(b, b->threads, b->cap);
    b->graph_launches = (int)(launches_so_far() - l1);
    count_launches(-b->graph_launches);  // counted at each replay
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, EGH_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
  }
  BCK(cudaGraphLaunch(b->graph, stream));
  count_launches(b->graph_launches);
  for (egh_ctx* c : b->ctxs) {  // the selective refinement's bounds of every mixed context
    const egh_status rs = refine_plan(c, stream);
    if (rs) return bfail(b, rs, c->err);
  }
  std::vector<int> stv(b->count);
  BCK(cudaMemcpyAsync(stv.data(), b->status, sizeof(int) * b->count, cudaMemcpyDeviceToHost, stream));
  BCK(cudaStreamSynchronize(stream));
  for (egh_ctx* c : b->ctxs) {
    const egh_status rs = refine_list(c);
    if (rs) return bfail(b, rs, c->err);
  }
  int o = 0;
  for (int i = 0; i < (int)b->ctxs.size(); ++i) {
    egh_ctx* c = b->ctxs[i];
    for (int k = 0; k < c->nf; ++k, ++o)
      if (stv[o]) {
        if (bad_ctx) *bad_ctx = i;
        if (bad_freq) *bad_freq = k;
        return bfail(b, EGH_ENOTPD, "Hessian " + std::to_string(k) + " of batch context " +
                                        std::to_string(i) + " not positive definite");
      }
  }
  for (egh_ctx* c : b->ctxs) c->state = ST_FACTORED;
  return EGH_OK;
}

const char* egh_batch_last_error(const egh_batch* b) {
  return b ? b->err.c_str() : egh_last_error(nullptr);
}

}  // extern "C"

namespace {

constexpr char kSetMagic[8] = {'E', 'G', 'H', 'Q', 'S', 'E', 'T', '1'};

void json_num(std::string& s, double v) {
  char b[40];
  snprintf(b, sizeof b, "%.17g", v);
  s += b;
}

template <class T>
void json_array(std::string& s, const std::vector<T>& v) {
  s += '[';
  for (size_t i = 0; i < v.size(); ++i) {
    if (i) s += ", ";
    json_num(s, (double)v[i]);
  }
  s += ']';
}

// The text after "key": in the header, or nullptr.
const char* json_find(const std::string& h, const char* key) {
  const std::string k = std::string("\"") + key + "\":";
  const size_t p = h.find(k);
  return p == std::string::npos ? nullptr : h.c_str() + p + k.size();
}

bool json_get(const std::string& h, const char* key, double* out) {
  const char* p = json_find(h, key);
  if (!p) return false;
  char* end = nullptr;
  *out = std::strtod(p, &end);
  return end != p;
}

bool json_get_array(const std::string& h, const char* key, std::vector<double>* out) {
  const char* p = json_find(h, key);
  if (!p) return false;
  while (*p == ' ') ++p;
  if (*p++ != '[') return false;
  out->clear();
  for (;;) {
    while (*p == ' ') ++p;
    if (*p == ']') return true;
    char* end = nullptr;
    const double v = std::strtod(p, &end);
    if (end == p) return false;
    out->push_back(v);
    p = end;
    while (*p == ' ') ++p;
    if (*p == ',') ++p;
    else if (*p != ']') return false;
  }
}

}  // namespace

extern "C" {

egh_status egh_save(egh_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(ctx, EGH_EINVAL, "NULL argument");
  CK(cudaSetDevice(ctx->dev));
  if (ctx->state < ST_FACTORED) return fail(ctx, EGH_ESTATE, "egh_save needs egh_factor first");
  const size_t n = (size_t)ctx->nf * ctx->nrec * ctx->nrec;
  std::vector<float2> q(n), l(n);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(q.data(), ctx->Qh, n * sizeof(float2), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(l.data(), ctx->Lh, n * sizeof(float2), cudaMemcpyDeviceToHost));
  const unsigned long long bytes = n * sizeof(float2);
  std::string h = "{\"format\": \"egh Hessian set\", \"version\": 1, \"nrec\": ";
  json_num(h, ctx->nrec);
  h += ", \"nfreq\": ";
  json_num(h, ctx->nf);
  h += ", \"freq_hz\": ";
  json_array(h, ctx->freqs);
  h += ", \"dt\": ";
  json_num(h, ctx->dt);
  h += ", \"nt\": ";
  json_num(h, ctx->nt);
  h += ", \"precision\": ";
  json_num(h, ctx->prec);
  h += ", \"mu\": ";
  json_num(h, ctx->mu);
  h += ", \"rec_iz\": ";
  json_array(h, ctx->rec_iz);
  h += ", \"rec_ix\": ";
  json_array(h, ctx->rec_ix);
  const std::string shape =
      "[" + std::to_string(ctx->nf) + ", " + std::to_string(ctx->nrec) + ", " + std::to_string(ctx->nrec) + "]";
  h += ", \"arrays\": [{\"name\": \"Q\", \"dtype\": \"complex64\", \"shape\": " + shape +
       ", \"offset\": 0}, {\"name\": \"L\", \"dtype\": \"complex64\", \"shape\": " + shape +
       ", \"offset\": " + std::to_string(bytes) + "}]}";
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(ctx, EGH_EINVAL, std::string("egh_save: cannot open ") + path);
  const unsigned long long hl = h.size();
  bool ok = std::fwrite(kSetMagic, 1, 8, f) == 8 && std::fwrite(&hl, 8, 1, f) == 1 &&
            std::fwrite(h.data(), 1, h.size(), f) == h.size() &&
            std::fwrite(q.data(), sizeof(float2), n, f) == n &&
            std::fwrite(l.data(), sizeof(float2), n, f) == n;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(ctx, EGH_EINVAL, std::string("egh_save: write failed: ") + path);
  return EGH_OK;
}

egh_status egh_load(egh_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(ctx, EGH_EINVAL, "NULL argument");
  CK(cudaSetDevice(ctx->dev));
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(ctx, EGH_EINVAL, std::string("egh_load: cannot open ") + path);
  auto bad = [&](const std::string& why) {
    std::fclose(f);
    return fail(ctx, EGH_EINVAL, "egh_load: " + why);
  };
  char magic[8];
  unsigned long long hl = 0;
  if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kSetMagic, 8) != 0)
    return bad("not a Hessian set file");
  if (std::fread(&hl, 8, 1, f) != 1 || hl == 0 || hl > (64ull << 20)) return bad("bad header length");
  std::string h(hl, '\0');
  if (std::fread(&h[0], 1, hl, f) != hl) return bad("truncated header");
  double nrec = 0, nfreq = 0, dt = 0, nt = 0, prec = 0, mu = 0;
  std::vector<double> fr, iz, ix;
  if (!json_get(h, "nrec", &nrec) || !json_get(h, "nfreq", &nfreq) || !json_get(h, "dt", &dt) ||
      !json_get(h, "nt", &nt) || !json_get(h, "precision", &prec) || !json_get(h, "mu", &mu) ||
      !json_get_array(h, "freq_hz", &fr) || !json_get_array(h, "rec_iz", &iz) ||
      !json_get_array(h, "rec_ix", &ix))
    return bad("incomplete header");
  if ((int)nrec != ctx->nrec || (int)nfreq != ctx->nf || (int)fr.size() != ctx->nf ||
      (int)iz.size() != ctx->nrec || (int)ix.size() != ctx->nrec)
    return bad("receiver or frequency count differs from the context's");
  for (int k = 0; k < ctx->nf; ++k)
    if (fr[k] != ctx->freqs[k]) return bad("frequencies differ from the context's");
  for (int r = 0; r < ctx->nrec; ++r)
    if ((int)iz[r] != ctx->rec_iz[r] || (int)ix[r] != ctx->rec_ix[r])
      return bad("receiver positions differ from the context's");
  if (dt != ctx->dt || (int)nt != ctx->nt) return bad("record (dt, nt) differs from the context's");
  if ((int)prec != ctx->prec) return bad("precision differs from the context's");
  if (!std::isfinite(mu) || mu < 0) return bad("mu is not a finite non-negative number");
  const size_t n = (size_t)ctx->nf * ctx->nrec * ctx->nrec;
  std::vector<float2> q(n);
  if (std::fread(q.data(), sizeof(float2), n, f) != n) return bad("truncated payload (Q)");
  {
    std::vector<float2> l(n);  // the saved factors: present, recomputed below
    if (std::fread(l.data(), sizeof(float2), n, f) != n) return bad("truncated payload (L)");
  }
  std::fclose(f);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(ctx->Qh, q.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
  ctx->mu = mu;
  ctx->st.mu = mu;
  ctx->state = ST_HESSIAN;
  int32_t bad_freq = -1;
  return egh_factor(ctx, &bad_freq, nullptr);
}

}  // extern "C"
