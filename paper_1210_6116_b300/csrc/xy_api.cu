// xy_api.cu -- host side of the C ABI declared in include/xy.h.
//
// The library owns only the small host handle; every device byte lives in the
// caller's workspace.  A sweep is five stream-ordered launches (bond+tile
// label, merge, compress, flip+measure, finalize) that read all per-sweep
// parameters (sweep counter, beta, axis) from device state, so a sequence of
// sweeps needs no host round trip and can be captured in a CUDA graph.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/xy.h"
#include "layout.cuh"
#include "sweep_kernels.cuh"
#include "launch.cuh"

using namespace xyk;

namespace {

thread_local char g_err[512] = "";

xy_status fail(xy_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

#define XY_CUDA(call)                                                       \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess)                                                  \
      return fail(XY_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

// Sets the calling thread's xy_last_error() message (used by xy_static.cu).
void xy_set_last_error_message(const char *msg) {
  snprintf(g_err, sizeof(g_err), "%s", msg);
}

struct xy_lattice {
  xy_config cfg;
  Layout lo;
  cudaStream_t stream;
  char *ws;
  LatDesc desc;       // host copy of the device descriptor
  LatDesc *d_desc;
  uint32_t *d_prefix;
  DevState *d_state;
  uint64_t enqueued;  // sweeps enqueued since xy_init
  bool write_labels = true;  // the next sweep stores canonical labels
  // how the next sweep is launched: K1's kCtl* bits (0: with k_finalize
  // after K4), and the k_finalize mode when ctl folds it (the call's last
  // sweep ends with the record-only finalize; the others launch none)
  uint32_t ctl = 0;
  bool fin_after = true;
  // CUDA graphs of kChunkSweeps sweeps from the middle of a call: [0] for
  // xy_sweep (folded finalize), [1] for xy_pcc_step (k_finalize after each
  // sweep).  Recorded on first use on a private stream and replayed on
  // `stream`; null until then, and again after a change of the descriptor
  // the kernels take.
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t chunk[2] = {nullptr, nullptr};
  uint64_t reported;  // sweeps already returned by xy_measure
  int sm_count;
  // kernel timing: 6 events per sweep bracket its kernels, the 5th being
  // k_finalize (the last two events are adjacent where the sweep launched
  // none)
  uint32_t prof;       // 0: off; k: time every k-th sweep
  uint64_t prof_count;  // sweeps launched since profiling was enabled
  bool prof_this;       // the sweep being launched is timed
  std::vector<cudaEvent_t> events;
  std::vector<uint8_t> ev_fin;  // per timed sweep: k_finalize was launched
  size_t ev_used;
};

namespace {

// records the next timing event of a profiled sweep (no-op otherwise)
cudaError_t mark(xy_lattice *h) {
  if (!h->prof_this) return cudaSuccess;
  if (h->ev_used == h->events.size()) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    h->events.push_back(e);
  }
  return cudaEventRecord(h->events[h->ev_used++], h->stream);
}

template <int TY, typename AT, bool EXACT, bool FULL>
cudaError_t launch_sweep_t(xy_lattice *h, cudaStream_t s) {
  h->prof_this = h->prof != 0 && h->prof_count++ % h->prof == 0;
  const uint32_t nw = h->lo.ntiles;
  cudaError_t e;
  if (h->desc.ragged) {
    e = cudaMemsetAsync(h->desc.coin, 0, (static_cast<size_t>(h->lo.L) * h->lo.L / 32 + 2) * 4, s);
    if (e != cudaSuccess) return e;
  }
  if ((e = mark(h)) != cudaSuccess) return e;
  const LatDesc *dd = h->d_desc;
  const uint32_t *pre = h->d_prefix;
  const LatDesc &one = h->desc;
  const uint32_t ctl = h->ctl, par = ctl & kCtlPar;
  const uint32_t nb1 = nw + ((ctl & kCtlDraw) ? 1u : 0u);  // + block 0 for the fold
  if ((e = launch_pdl(k_bond_label<TY, AT, EXACT, false, FULL, true>, nb1, kThreads,
                      bond_label_smem<TY>(), s, dd, pre, 1u, nw, ctl, one)) != cudaSuccess)
    return e;
  if ((e = mark(h)) != cudaSuccess) return e;
  const uint64_t items = static_cast<uint64_t>(nw) * (TY + 32);
  const uint64_t eb = (items + kThreads - 1) / kThreads;
  if ((e = launch_pdl(k_merge<TY, FULL, true>, static_cast<uint32_t>(eb), kThreads, 0, s, dd,
                      pre, 1u, nw, one)) != cudaSuccess)
    return e;
  if ((e = mark(h)) != cudaSuccess) return e;
  if ((e = launch_pdl(k_compress<TY, true>, compress_blocks(nw), kThreads, 0, s, dd, pre, 1u, nw,
                      one)) != cudaSuccess)
    return e;
  if ((e = mark(h)) != cudaSuccess) return e;
  // the extended K4 for chik sums or Wolff; canonical labels only for the
  // last sweep of an xy_sweep / xy_pcc_step call
  const bool ext = h->desc.xi || h->desc.wolff;
  if (ext && h->write_labels)
    e = launch_pdl(k_flip_measure<TY, AT, false, true, true, FULL, true>, nw, kThreads,
                   flip_smem<TY>(), s, dd, pre, 1u, nw, par, one);
  else if (ext)
    e = launch_pdl(k_flip_measure<TY, AT, false, true, false, FULL, true>, nw, kThreads,
                   flip_smem<TY>(), s, dd, pre, 1u, nw, par, one);
  else if (h->write_labels)
    e = launch_pdl(k_flip_measure<TY, AT, false, false, true, FULL, true>, nw, kThreads,
                   flip_smem<TY>(), s, dd, pre, 1u, nw, par, one);
  else
    e = launch_pdl(k_flip_measure<TY, AT, false, false, false, FULL, true>, nw, kThreads,
                   flip_smem<TY>(), s, dd, pre, 1u, nw, par, one);
  if (e != cudaSuccess) return e;
  if ((e = mark(h)) != cudaSuccess) return e;
  if (h->fin_after) {
    const uint32_t mode = (ctl & kCtlDraw) ? (kFinRecord | par) : 0u;
    if ((e = launch_pdl(k_finalize, 1u, kFinalizeThreads, 0, s, dd, 1u, mode)) != cudaSuccess)
      return e;
  }
  if (h->prof_this) h->ev_fin.push_back(h->fin_after ? 1 : 0);
  if ((e = mark(h)) != cudaSuccess) return e;
  return cudaGetLastError();
}

// whole tiles only (L a multiple of 32 and of TY): the FULL kernels
template <int TY, typename AT, bool EXACT>
cudaError_t launch_exact_full(xy_lattice *h, cudaStream_t s) {
  const bool full = h->lo.L % 32u == 0u && h->lo.L % static_cast<uint32_t>(TY) == 0u;
  return full ? launch_sweep_t<TY, AT, EXACT, true>(h, s)
              : launch_sweep_t<TY, AT, EXACT, false>(h, s);
}

template <int TY, typename AT, bool EXACT>
cudaError_t set_attrs_t() {
  cudaError_t e = cudaFuncSetAttribute(k_bond_label<TY, AT, EXACT, false, false, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(bond_label_smem<TY>()));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_bond_label<TY, AT, EXACT, false, true, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(bond_label_smem<TY>()));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_bond_label<TY, AT, EXACT, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(bond_label_smem<TY>()));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_flip_measure<TY, AT, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(flip_smem<TY>()));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_flip_measure<TY, AT, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(flip_smem<TY>()));
}

template <int TY, typename AT>
cudaError_t dispatch_exact(xy_lattice *h, bool attrs, cudaStream_t s) {
  if (h->cfg.threshold_mode == XY_THR_F64)
    return attrs ? set_attrs_t<TY, AT, true>() : launch_exact_full<TY, AT, true>(h, s);
  return attrs ? set_attrs_t<TY, AT, false>() : launch_exact_full<TY, AT, false>(h, s);
}

template <typename AT>
cudaError_t dispatch_ty(xy_lattice *h, bool attrs, cudaStream_t s) {
  switch (h->lo.TY) {
    case 16: return dispatch_exact<16, AT>(h, attrs, s);
    case 32: return dispatch_exact<32, AT>(h, attrs, s);
    case 64: return dispatch_exact<64, AT>(h, attrs, s);
    default: return dispatch_exact<128, AT>(h, attrs, s);
  }
}

cudaError_t dispatch_dtype(xy_lattice *h, bool attrs, cudaStream_t s) {
  switch (h->cfg.angle_dtype) {
    case XY_F32: return dispatch_ty<float>(h, attrs, s);
    case XY_F16: return dispatch_ty<__half>(h, attrs, s);
    default: return dispatch_ty<uint16_t>(h, attrs, s);
  }
}

cudaError_t launch_sweep(xy_lattice *h, cudaStream_t s) { return dispatch_dtype(h, false, s); }

cudaError_t set_attrs(xy_lattice *h) { return dispatch_dtype(h, true, nullptr); }

// Sweeps per replay of the chunk graph.  Even, so that every chunk starts
// on the same parameter slot.  With K1 and K4 triggering their dependent
// launches after their waits, chunks of 8 to 64 sweeps time within 0.3 us
// per sweep of each other at L = 256 .. 4096.
constexpr uint32_t kChunkSweeps = 16;

// Sweep k of an xy_sweep call: the parameter slot k & 1, the record of the
// previous sweep from k = 1 on, k_finalize only after the last sweep.
void set_fold_sweep(xy_lattice *h, uint32_t k, uint32_t n) {
  h->write_labels = k + 1 == n;  // labels of the call's last sweep
  h->ctl = (k & 1u) | kCtlDraw | (k ? kCtlRecord : 0u);
  h->fin_after = k + 1 == n;
}

// Sweep k of an xy_pcc_step call: k_finalize after every sweep (the next
// beta depends on the record), labels of the last sweep.
void set_pcc_sweep(xy_lattice *h, uint32_t k, uint32_t n) {
  h->write_labels = k + 1 == n;
  h->ctl = 0u;
  h->fin_after = true;
}

void drop_chunk(xy_lattice *h) {
  for (cudaGraphExec_t &g : h->chunk) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

// Record chunk graph `which` (0: xy_sweep, 1: xy_pcc_step): kChunkSweeps
// sweeps from an odd sweep index of a call, none of them the call's last.
// The kernels take the descriptor by value and the workspace pointers, all
// fixed for the handle; a change of the descriptor drops the graphs
// (drop_chunk).
cudaError_t record_chunk(xy_lattice *h, int which) {
  cudaError_t e;
  if (!h->cap_stream &&
      (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return e;
  if ((e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return e;
  // no timing events inside the graph: profiling is off while recording
  const uint32_t prof = h->prof;
  const uint64_t prof_count = h->prof_count;
  h->prof = 0;
  cudaError_t le = cudaSuccess;
  for (uint32_t j = 0; j < kChunkSweeps && le == cudaSuccess; ++j) {
    if (which == 0) set_fold_sweep(h, j + 1u, kChunkSweeps + 2u);
    else set_pcc_sweep(h, j + 1u, kChunkSweeps + 2u);
    le = launch_sweep(h, h->cap_stream);
  }
  h->prof = prof;
  h->prof_count = prof_count;
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(h->cap_stream, &g);  // ends the capture even after a failed launch
  if (le != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le != cudaSuccess ? le : e;
  }
  e = cudaGraphInstantiate(&h->chunk[which], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) h->chunk[which] = nullptr;
  return e;
}

// Enqueue sweeps 0 .. n-1 of a call (which = 0: xy_sweep, 1: xy_pcc_step).
// Runs of kChunkSweeps sweeps from an odd index that end before the call's
// last sweep replay chunk graph `which`, unless the stream is being
// captured by the caller or xy_profile would time a sweep of the run; the
// others are launched directly.  The graph is recorded by the first call of
// its kind, however short: recording takes the host ~1 ms, which a later,
// longer call would otherwise spend with the GPU waiting.
cudaError_t enqueue_sweeps(xy_lattice *h, uint32_t n, int which) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(h->stream, &cap);
  if (e != cudaSuccess) return e;
  const bool graphs = cap == cudaStreamCaptureStatusNone;
  if (graphs && n && !h->chunk[which] && (e = record_chunk(h, which)) != cudaSuccess) return e;
  for (uint32_t k = 0; k < n;) {
    const bool odd_middle = (k & 1u) && n - 1u - k >= kChunkSweeps;
    bool timed = false;  // a sweep of the run would be profiled
    for (uint32_t j = 0; odd_middle && h->prof && j < kChunkSweeps && !timed; ++j)
      timed = (h->prof_count + j) % h->prof == 0;
    if (graphs && odd_middle && !timed) {
      if ((e = cudaGraphLaunch(h->chunk[which], h->stream)) != cudaSuccess) return e;
      h->prof_count += kChunkSweeps;
      k += kChunkSweeps;
      continue;
    }
    if (which == 0) set_fold_sweep(h, k, n);
    else set_pcc_sweep(h, k, n);
    if ((e = launch_sweep(h, h->stream)) != cudaSuccess) return e;
    ++k;
  }
  return cudaSuccess;
}

// labeling only, from the bond planes already in the workspace
template <int TY>
cudaError_t launch_label_only_t(xy_lattice *h) {
  const uint32_t nw = h->lo.ntiles;
  cudaStream_t s = h->stream;
  k_bond_label<TY, float, true, true>
      <<<nw, kThreads, bond_label_smem<TY>(), s>>>(h->d_desc, h->d_prefix, 1, nw, 0u, LatDesc{});
  const uint64_t items = static_cast<uint64_t>(nw) * (TY + 32);
  const uint32_t eb = static_cast<uint32_t>((items + kThreads - 1) / kThreads);
  k_merge<TY><<<eb, kThreads, 0, s>>>(h->d_desc, h->d_prefix, 1, nw, LatDesc{});
  k_compress<TY><<<compress_blocks(nw), kThreads, 0, s>>>(h->d_desc, h->d_prefix, 1, nw,
                                                          LatDesc{});
  k_flip_measure<TY, float, true>
      <<<nw, kThreads, flip_smem<TY>(), s>>>(h->d_desc, h->d_prefix, 1, nw, 0u, LatDesc{});
  return cudaGetLastError();
}

cudaError_t launch_label_only(xy_lattice *h) {
  if (h->cfg.angle_dtype != XY_F32) {
    // the label-only kernels are dtype-agnostic; make sure their attributes
    // are set even when the lattice itself stores FP16 or u16 angles
    cudaError_t e;
    switch (h->lo.TY) {
      case 16: e = set_attrs_t<16, float, true>(); break;
      case 32: e = set_attrs_t<32, float, true>(); break;
      case 64: e = set_attrs_t<64, float, true>(); break;
      default: e = set_attrs_t<128, float, true>(); break;
    }
    if (e != cudaSuccess) return e;
  }
  switch (h->lo.TY) {
    case 16: return launch_label_only_t<16>(h);
    case 32: return launch_label_only_t<32>(h);
    case 64: return launch_label_only_t<64>(h);
    default: return launch_label_only_t<128>(h);
  }
}

// Report the lattice's device error word and clear it: an error is reported
// once, and the handle stays usable (the kernels that set the word finished
// their launches; the labels of the affected sweep are not meaningful).
xy_status check_device_error(xy_lattice *h) {
  uint32_t err = 0;
  XY_CUDA(cudaMemcpy(&err, &h->d_state->err, sizeof(err), cudaMemcpyDeviceToHost));
  if (err) XY_CUDA(cudaMemset(&h->d_state->err, 0, sizeof(err)));
  return device_error_status(err);
}

}  // namespace

// Sampled state for xy_get_sites: angle (raw bits of the storage format),
// label and the two bond bits of each listed site.  16-bit formats (FP16 and
// u16) are copied as their bits.
template <typename AT>
__global__ void k_gather_sites(LatDesc d, uint32_t TY, const uint64_t *__restrict__ sites,
                               uint32_t n, uint32_t cur, AT *theta_out, uint32_t *label_out,
                               uint8_t *bonds_out) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint64_t i = sites[k];
  const uint32_t x = static_cast<uint32_t>(i % d.L), y = static_cast<uint32_t>(i / d.L);
  theta_out[k] = static_cast<const AT *>(d.theta[cur])[i];
  label_out[k] = d.label[i];
  const uint64_t w = static_cast<uint64_t>((y / TY) * d.ntx + x / 32u) * TY + y % TY;
  bonds_out[k] = static_cast<uint8_t>(((d.rplane[w] >> (x & 31u)) & 1u) |
                                      (((d.dplane[w] >> (x & 31u)) & 1u) << 1));
}

// cos and sin of the angles i0 .. i0 + n - 1 with the observables' routine
template <typename AT>
__global__ void k_spins(LatDesc d, uint32_t cur, uint64_t i0, uint64_t n, float *cs,
                        float *sn) {
  const AT *th = static_cast<const AT *>(d.theta[cur]);
  for (uint64_t k = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n;
       k += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    float s, c;
    sin_cos<AT>(load_angle(th, i0 + k), &s, &c);
    cs[k] = c;
    sn[k] = s;
  }
}

extern "C" {

const char *xy_last_error(void) { return g_err; }

xy_status xy_workspace_size(const xy_config *cfg, size_t *bytes) {
  if (!bytes) return fail(XY_EINVAL, "bytes is NULL");
  Layout lo;
  xy_status s = make_layout(cfg, &lo);
  if (s != XY_OK) return s;
  *bytes = lo.total;
  return XY_OK;
}

xy_status xy_init(const xy_config *cfg, void *d_workspace, size_t bytes,
                  void *cuda_stream, xy_lattice **out) {
  if (!out) return fail(XY_EINVAL, "out is NULL");
  *out = nullptr;
  Layout lo;
  xy_status st = make_layout(cfg, &lo);
  if (st != XY_OK) return st;
  if (!d_workspace) return fail(XY_EINVAL, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256)
    return fail(XY_EINVAL, "workspace must be 256-byte aligned");
  if (bytes < lo.total)
    return fail(XY_ENOMEM, "workspace of %zu bytes, %zu needed", bytes, lo.total);
  xy_lattice *h = new (std::nothrow) xy_lattice();
  if (!h) return fail(XY_ENOMEM, "host allocation failed");
  h->cfg = *cfg;
  h->lo = lo;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->ws = static_cast<char *>(d_workspace);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete h;
    return fail(XY_ECUDA, "no CUDA device");
  }
  h->desc = make_desc(cfg, lo, h->ws);
  LatDesc &d = h->desc;
  h->d_desc = reinterpret_cast<LatDesc *>(h->ws + lo.off_desc);
  h->d_prefix = reinterpret_cast<uint32_t *>(h->ws + lo.off_prefix);
  h->d_state = d.st;
  const uint32_t prefix[2] = {0u, lo.ntiles};
  auto bail = [&](const char *what, cudaError_t e) {
    delete h;
    return fail(XY_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = set_attrs(h)) != cudaSuccess) return bail("cudaFuncSetAttribute", e);
  if ((e = cudaMemcpyAsync(h->d_desc, &h->desc, sizeof(LatDesc), cudaMemcpyHostToDevice,
                           h->stream)) != cudaSuccess)
    return bail("descriptor upload", e);
  if ((e = cudaMemcpyAsync(h->d_prefix, prefix, sizeof(prefix), cudaMemcpyHostToDevice,
                           h->stream)) != cudaSuccess)
    return bail("prefix upload", e);
  if ((e = cudaMemsetAsync(d.acc, 0, sizeof(long long) * kSlots * kAccStride, h->stream)) !=
      cudaSuccess)
    return bail("accumulator reset", e);
  if ((e = cudaMemsetAsync(d.coin, 0, (static_cast<size_t>(lo.L) * lo.L / 32 + 2) * 4,
                           h->stream)) != cudaSuccess)
    return bail("coin reset", e);
  k_init_state<<<1, 1, 0, h->stream>>>(d, cfg->beta, cfg->angle_dtype == XY_U16 ? 1u : 0u);
  k_init_wave<<<(lo.L + 255) / 256, 256, 0, h->stream>>>(d);
  const uint64_t n = static_cast<uint64_t>(lo.L) * lo.L;
  const uint32_t blocks = static_cast<uint32_t>(
      std::min<uint64_t>((n + 255) / 256, static_cast<uint64_t>(h->sm_count) * 16));
  if (cfg->angle_dtype == XY_F32)
    k_init_angles<float><<<blocks, 256, 0, h->stream>>>(d, cfg->start);
  else if (cfg->angle_dtype == XY_F16)
    k_init_angles<__half><<<blocks, 256, 0, h->stream>>>(d, cfg->start);
  else
    k_init_angles<uint16_t><<<blocks, 256, 0, h->stream>>>(d, cfg->start);
  if ((e = cudaGetLastError()) != cudaSuccess) return bail("init launch", e);
  // the host copies above read stack memory: finish them before returning
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail("init sync", e);
  *out = h;
  return XY_OK;
}

// NVTX range around the host work of an API call (no cost without a tool
// attached): a profiler's timeline shows which call enqueued which kernels.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

xy_status xy_sweep(xy_lattice *h, uint32_t n_sweeps) {
  if (!h) return fail(XY_EINVAL, "handle is NULL");
  NvtxRange range("xy_sweep");
  k_set_pcc<<<1, 1, 0, h->stream>>>(h->d_state, 0u, 0.0, 0.0, 0u, 1u);
  // fixed beta: sweep k keeps its parameters in slot k & 1, its K1 draws the
  // next sweep's and appends the previous sweep's record (kCtlDraw), and only
  // the last sweep is followed by k_finalize (the last record)
  XY_CUDA(enqueue_sweeps(h, n_sweeps, 0));
  XY_CUDA(cudaGetLastError());
  h->enqueued += n_sweeps;
  return XY_OK;
}

xy_status xy_pcc_step(xy_lattice *h, const xy_pcc_params *p, uint32_t n_sweeps) {
  if (!h) return fail(XY_EINVAL, "handle is NULL");
  if (!p) return fail(XY_EINVAL, "params is NULL");
  if (p->block == 0) return fail(XY_EINVAL, "block must be >= 1");
  if (!(p->dbeta0 >= 0.0) || !std::isfinite(p->dbeta0) || !std::isfinite(p->target))
    return fail(XY_EINVAL, "dbeta0 must be finite and >= 0, target finite");
  NvtxRange range("xy_pcc_step");
  k_set_pcc<<<1, 1, 0, h->stream>>>(h->d_state, 1u, p->target, p->dbeta0, p->halve_every,
                                    p->block);
  // the next sweep's beta depends on this sweep's record: k_finalize after
  // every sweep
  XY_CUDA(enqueue_sweeps(h, n_sweeps, 1));
  XY_CUDA(cudaGetLastError());
  h->enqueued += n_sweeps;
  return XY_OK;
}

xy_status xy_measure(xy_lattice *h, xy_obs *out, uint32_t max_records, uint32_t *n_out,
                     int sync) {
  if (!h || !n_out) return fail(XY_EINVAL, "NULL argument");
  *n_out = 0;
  if (max_records && !out) return fail(XY_EINVAL, "out is NULL");
  if (sync) {
    XY_CUDA(cudaStreamSynchronize(h->stream));
    xy_status s = check_device_error(h);
    if (s != XY_OK) return s;
  }
  const uint64_t pending = h->enqueued - h->reported;
  const uint64_t avail = std::min<uint64_t>(pending, h->lo.rec_cap);
  const uint64_t take = std::min<uint64_t>(avail, max_records);
  const uint64_t first = h->enqueued - take;  // sweep index of the first record returned
  for (uint64_t k = 0; k < take;) {
    const uint64_t slot = (first + k) % h->lo.rec_cap;
    const uint64_t run = std::min<uint64_t>(take - k, h->lo.rec_cap - slot);
    XY_CUDA(cudaMemcpy(out + k, h->desc.rec + slot, run * sizeof(xy_obs),
                       cudaMemcpyDeviceToHost));
    k += run;
  }
  h->reported = h->enqueued;
  *n_out = static_cast<uint32_t>(take);
  return XY_OK;
}

xy_status xy_get_state(xy_lattice *h, double *beta, uint64_t *sweep) {
  if (!h) return fail(XY_EINVAL, "handle is NULL");
  XY_CUDA(cudaStreamSynchronize(h->stream));
  DevState s;
  XY_CUDA(cudaMemcpy(&s, h->d_state, sizeof(s), cudaMemcpyDeviceToHost));
  if (beta) *beta = s.p[0].beta;
  if (sweep) *sweep = s.p[0].t;
  return XY_OK;
}

xy_status xy_destroy(xy_lattice *h) {
  if (!h) return fail(XY_EINVAL, "handle is NULL");
  cudaStreamSynchronize(h->stream);
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  drop_chunk(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
  return XY_OK;
}

namespace {
// the copies and sweeps of xy_run_host, enqueued on the lattice's stream
xy_status run_host_enqueue(xy_lattice *h, const void *host_angles_in, uint32_t n_sweeps,
                           xy_obs *host_obs, void *host_angles_out) {
  if (!h) return fail(XY_EINVAL, "handle is NULL");
  NvtxRange range("xy_run_host");
  const size_t ab = static_cast<size_t>(h->lo.L) * h->lo.L * h->lo.esize;
  // the angle buffer the next sweep reads is theta[cur]; cur flips once per
  // sweep, so it is known on the host from the number of sweeps enqueued
  const uint32_t cur0 = static_cast<uint32_t>(h->enqueued & 1u);
  if (host_angles_in)
    XY_CUDA(cudaMemcpyAsync(h->desc.theta[cur0], host_angles_in, ab, cudaMemcpyHostToDevice,
                            h->stream));
  xy_status s = xy_sweep(h, n_sweeps);
  if (s != XY_OK) return s;
  const uint32_t cur1 = static_cast<uint32_t>(h->enqueued & 1u);
  if (host_obs && n_sweeps) {
    const uint64_t take = std::min<uint64_t>(n_sweeps, h->lo.rec_cap);
    const uint64_t first = h->enqueued - take;
    for (uint64_t k = 0; k < take;) {
      const uint64_t slot = (first + k) % h->lo.rec_cap;
      const uint64_t run = std::min<uint64_t>(take - k, h->lo.rec_cap - slot);
      XY_CUDA(cudaMemcpyAsync(host_obs + (n_sweeps - take) + k, h->desc.rec + slot,
                              run * sizeof(xy_obs), cudaMemcpyDeviceToHost, h->stream));
      k += run;
    }
    h->reported = h->enqueued;
  }
  if (host_angles_out)
    XY_CUDA(cudaMemcpyAsync(host_angles_out, h->desc.theta[cur1], ab, cudaMemcpyDeviceToHost,
                            h->stream));
  return XY_OK;
}
}  // namespace

xy_status xy_run_host(xy_lattice *h, const void *host_angles_in, uint32_t n_sweeps,
                      xy_obs *host_obs, void *host_angles_out) {
  const xy_status s = run_host_enqueue(h, host_angles_in, n_sweeps, host_obs, host_angles_out);
  if (s != XY_OK) return s;
  XY_CUDA(cudaStreamSynchronize(h->stream));
  return check_device_error(h);
}

xy_status xy_run_host_async(xy_lattice *h, const void *host_angles_in, uint32_t n_sweeps,
                            xy_obs *host_obs, void *host_angles_out) {
  return run_host_enqueue(h, host_angles_in, n_sweeps, host_obs, host_angles_out);
}

xy_status xy_sync(xy_lattice *h) {
  if (!h) return fail(XY_EINVAL, "handle is NULL");
  XY_CUDA(cudaStreamSynchronize(h->stream));
  return check_device_error(h);
}

xy_status xy_profile(xy_lattice *h, int enable) {
  if (!h) return fail(XY_EINVAL, "handle is NULL");
  XY_CUDA(cudaStreamSynchronize(h->stream));
  if (enable < 0) return fail(XY_EINVAL, "enable must be >= 0");
  h->prof = static_cast<uint32_t>(enable);
  h->prof_count = 0;
  h->ev_used = 0;
  h->ev_fin.clear();
  return XY_OK;
}

xy_status xy_profile_read(xy_lattice *h, xy_kernel_times *out) {
  if (!h || !out) return fail(XY_EINVAL, "NULL argument");
  XY_CUDA(cudaStreamSynchronize(h->stream));
  std::memset(out, 0, sizeof(*out));
  // events come in groups of 6 per sweep
  for (size_t base = 0, j = 0; base + 6 <= h->ev_used; base += 6, ++j) {
    for (int k = 0; k < XY_NUM_KERNELS; ++k) {
      if (k == XY_NUM_KERNELS - 1 && !h->ev_fin[j]) continue;  // no k_finalize
      float ms = 0.0f;
      XY_CUDA(cudaEventElapsedTime(&ms, h->events[base + k], h->events[base + k + 1]));
      out->ms[k] += ms;
      out->launches[k] += 1;
    }
  }
  return XY_OK;
}

xy_status xy_get_angles(xy_lattice *h, void *host_dst) {
  if (!h || !host_dst) return fail(XY_EINVAL, "NULL argument");
  XY_CUDA(cudaStreamSynchronize(h->stream));
  DevState s;
  XY_CUDA(cudaMemcpy(&s, h->d_state, sizeof(s), cudaMemcpyDeviceToHost));
  const size_t bytes = static_cast<size_t>(h->lo.L) * h->lo.L * h->lo.esize;
  XY_CUDA(cudaMemcpy(host_dst, h->desc.theta[s.p[0].cur], bytes, cudaMemcpyDeviceToHost));
  return XY_OK;
}

xy_status xy_get_spins(xy_lattice *h, float *host_cos, float *host_sin) {
  if (!h) return fail(XY_EINVAL, "NULL lattice");
  XY_CUDA(cudaStreamSynchronize(h->stream));
  DevState st;
  XY_CUDA(cudaMemcpy(&st, h->d_state, sizeof(st), cudaMemcpyDeviceToHost));
  const uint64_t n = static_cast<uint64_t>(h->lo.L) * h->lo.L;
  const uint64_t chunk = std::min<uint64_t>(n, 1ull << 22);  // 2 x 16 MiB
  float *buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, chunk * 2 * sizeof(float));
  for (uint64_t i0 = 0; e == cudaSuccess && i0 < n; i0 += chunk) {
    const uint64_t m = std::min(chunk, n - i0);
    const uint32_t blocks = static_cast<uint32_t>(std::min<uint64_t>((m + 255) / 256, static_cast<uint64_t>(h->sm_count) * 16));
    if (h->cfg.angle_dtype == XY_F32)
      k_spins<float><<<blocks, 256, 0, h->stream>>>(h->desc, st.p[0].cur, i0, m, buf, buf + chunk);
    else if (h->cfg.angle_dtype == XY_F16)
      k_spins<__half><<<blocks, 256, 0, h->stream>>>(h->desc, st.p[0].cur, i0, m, buf, buf + chunk);
    else
      k_spins<uint16_t><<<blocks, 256, 0, h->stream>>>(h->desc, st.p[0].cur, i0, m, buf, buf + chunk);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess && host_cos)
      e = cudaMemcpy(host_cos + i0, buf, m * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && host_sin)
      e = cudaMemcpy(host_sin + i0, buf + chunk, m * sizeof(float), cudaMemcpyDeviceToHost);
  }
  cudaFree(buf);
  if (e != cudaSuccess) return fail(XY_ECUDA, "xy_get_spins: %s", cudaGetErrorString(e));
  return XY_OK;
}

xy_status xy_set_angles(xy_lattice *h, const void *host_src) {
  if (!h || !host_src) return fail(XY_EINVAL, "NULL argument");
  const uint64_t n = static_cast<uint64_t>(h->lo.L) * h->lo.L;
  const float two_pi = 6.2831854820251465f;
  if (h->lo.esize == 4) {
    const float *a = static_cast<const float *>(host_src);
    for (uint64_t i = 0; i < n; ++i)
      if (!(a[i] >= 0.0f && a[i] < two_pi))
        return fail(XY_EINVAL, "angle %llu = %g outside [0, 2pi)",
                    static_cast<unsigned long long>(i), a[i]);
  } else if (h->cfg.angle_dtype == XY_F16) {
    const __half_raw *a = static_cast<const __half_raw *>(host_src);
    for (uint64_t i = 0; i < n; ++i) {
      const float v = __half2float(__half(a[i]));
      if (!(v >= 0.0f && v < two_pi))
        return fail(XY_EINVAL, "angle %llu = %g outside [0, 2pi)",
                    static_cast<unsigned long long>(i), v);
    }
  }  // u16: every q in 0..65535 is an angle in [0, 2pi)
  XY_CUDA(cudaStreamSynchronize(h->stream));
  DevState s;
  XY_CUDA(cudaMemcpy(&s, h->d_state, sizeof(s), cudaMemcpyDeviceToHost));
  XY_CUDA(cudaMemcpy(h->desc.theta[s.p[0].cur], host_src, n * h->lo.esize, cudaMemcpyHostToDevice));
  return XY_OK;
}

xy_status xy_get_bonds(xy_lattice *h, uint8_t *host_right, uint8_t *host_down) {
  if (!h || !host_right || !host_down) return fail(XY_EINVAL, "NULL argument");
  XY_CUDA(cudaStreamSynchronize(h->stream));
  const size_t words = static_cast<size_t>(h->lo.ntiles) * h->lo.TY;
  std::vector<uint32_t> R(words), D(words);
  XY_CUDA(cudaMemcpy(R.data(), h->desc.rplane, words * 4, cudaMemcpyDeviceToHost));
  XY_CUDA(cudaMemcpy(D.data(), h->desc.dplane, words * 4, cudaMemcpyDeviceToHost));
  const uint32_t L = h->lo.L, TY = h->lo.TY;
  for (uint32_t tile = 0; tile < h->lo.ntiles; ++tile) {
    const uint32_t x0 = (tile % h->lo.ntx) * 32, y0 = (tile / h->lo.ntx) * TY;
    const uint32_t w = std::min(32u, L - x0), hh = std::min(TY, L - y0);
    for (uint32_t r = 0; r < hh; ++r)
      for (uint32_t c = 0; c < w; ++c) {
        const size_t i = static_cast<size_t>(y0 + r) * L + x0 + c;
        host_right[i] = (R[static_cast<size_t>(tile) * TY + r] >> c) & 1u;
        host_down[i] = (D[static_cast<size_t>(tile) * TY + r] >> c) & 1u;
      }
  }
  return XY_OK;
}

xy_status xy_get_labels(xy_lattice *h, uint32_t *host_dst) {
  if (!h || !host_dst) return fail(XY_EINVAL, "NULL argument");
  XY_CUDA(cudaStreamSynchronize(h->stream));
  XY_CUDA(cudaMemcpy(host_dst, h->desc.label, static_cast<size_t>(h->lo.L) * h->lo.L * 4,
                     cudaMemcpyDeviceToHost));
  return XY_OK;
}

xy_status xy_get_sites(xy_lattice *h, const uint64_t *host_sites, uint32_t n,
                       void *host_theta, uint32_t *host_label, uint8_t *host_bonds) {
  if (!h || (n > 0 && !host_sites)) return fail(XY_EINVAL, "NULL argument");
  if (n == 0) return XY_OK;
  const uint64_t N = static_cast<uint64_t>(h->lo.L) * h->lo.L;
  for (uint32_t k = 0; k < n; ++k)
    if (host_sites[k] >= N)
      return fail(XY_EINVAL, "site %llu outside 0..N-1", static_cast<unsigned long long>(host_sites[k]));
  XY_CUDA(cudaStreamSynchronize(h->stream));
  DevState st;
  XY_CUDA(cudaMemcpy(&st, h->d_state, sizeof(st), cudaMemcpyDeviceToHost));
  const size_t es = h->lo.esize;
  const size_t off_t = static_cast<size_t>(n) * 8, off_l = off_t + align_up(n * es, 16),
               off_b = off_l + static_cast<size_t>(n) * 4, bytes = off_b + n;
  char *buf = nullptr;
  XY_CUDA(cudaMalloc(&buf, bytes));
  cudaError_t e = cudaMemcpy(buf, host_sites, static_cast<size_t>(n) * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const uint64_t *sites = reinterpret_cast<const uint64_t *>(buf);
    uint32_t *lab = reinterpret_cast<uint32_t *>(buf + off_l);
    uint8_t *bd = reinterpret_cast<uint8_t *>(buf + off_b);
    const uint32_t blocks = (n + 255) / 256;
    if (h->cfg.angle_dtype == XY_F32)
      k_gather_sites<float><<<blocks, 256>>>(h->desc, h->lo.TY, sites, n, st.p[0].cur,
                                             reinterpret_cast<float *>(buf + off_t), lab, bd);
    else
      k_gather_sites<uint16_t><<<blocks, 256>>>(h->desc, h->lo.TY, sites, n, st.p[0].cur,
                                                reinterpret_cast<uint16_t *>(buf + off_t), lab, bd);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && host_theta) e = cudaMemcpy(host_theta, buf + off_t, n * es, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && host_label) e = cudaMemcpy(host_label, lab, static_cast<size_t>(n) * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && host_bonds) e = cudaMemcpy(host_bonds, bd, n, cudaMemcpyDeviceToHost);
  }
  cudaFree(buf);
  if (e != cudaSuccess) return fail(XY_ECUDA, "xy_get_sites: %s", cudaGetErrorString(e));
  return XY_OK;
}

xy_status xy_label_bonds(xy_lattice *h, const uint8_t *host_right, const uint8_t *host_down,
                         uint32_t *host_labels) {
  if (!h || !host_right || !host_down || !host_labels) return fail(XY_EINVAL, "NULL argument");
  const uint32_t L = h->lo.L, TY = h->lo.TY;
  const size_t words = static_cast<size_t>(h->lo.ntiles) * TY;
  std::vector<uint32_t> R(words, 0u), D(words, 0u);
  for (uint32_t tile = 0; tile < h->lo.ntiles; ++tile) {
    const uint32_t x0 = (tile % h->lo.ntx) * 32, y0 = (tile / h->lo.ntx) * TY;
    const uint32_t w = std::min(32u, L - x0), hh = std::min(TY, L - y0);
    for (uint32_t r = 0; r < hh; ++r)
      for (uint32_t c = 0; c < w; ++c) {
        const size_t i = static_cast<size_t>(y0 + r) * L + x0 + c;
        if (host_right[i] > 1 || host_down[i] > 1)
          return fail(XY_EINVAL, "bond bytes must be 0 or 1");
        R[static_cast<size_t>(tile) * TY + r] |= static_cast<uint32_t>(host_right[i]) << c;
        D[static_cast<size_t>(tile) * TY + r] |= static_cast<uint32_t>(host_down[i]) << c;
      }
  }
  XY_CUDA(cudaStreamSynchronize(h->stream));
  XY_CUDA(cudaMemcpy(h->desc.rplane, R.data(), words * 4, cudaMemcpyHostToDevice));
  XY_CUDA(cudaMemcpy(h->desc.dplane, D.data(), words * 4, cudaMemcpyHostToDevice));
  XY_CUDA(launch_label_only(h));
  XY_CUDA(cudaStreamSynchronize(h->stream));
  xy_status s = check_device_error(h);
  if (s != XY_OK) return s;
  XY_CUDA(cudaMemcpy(host_labels, h->desc.label, static_cast<size_t>(L) * L * 4,
                     cudaMemcpyDeviceToHost));
  return XY_OK;
}

xy_status xy_build_arch(int *binary_version) {
  if (!binary_version) return fail(XY_EINVAL, "binary_version is NULL");
  cudaFuncAttributes a{};
  XY_CUDA(cudaFuncGetAttributes(&a, k_finalize));
  *binary_version = a.binaryVersion;
  return XY_OK;
}

xy_status xy_set_loop_bound(xy_lattice *h, uint32_t cap) {
  if (!h) return fail(XY_EINVAL, "handle is NULL");
  XY_CUDA(cudaStreamSynchronize(h->stream));
  h->desc.find_cap = cap ? cap : kFindCap;
  drop_chunk(h);  // the graph holds the old descriptor
  XY_CUDA(cudaMemcpy(h->d_desc, &h->desc, sizeof(LatDesc), cudaMemcpyHostToDevice));
  return XY_OK;
}

xy_status xy_set_link_cap(xy_lattice *h, uint32_t cap) {
  if (!h) return fail(XY_EINVAL, "handle is NULL");
  XY_CUDA(cudaStreamSynchronize(h->stream));
  const uint32_t full = h->lo.TY + 32u;
  h->desc.link_cap = (cap == 0u || cap > full) ? full : cap;
  drop_chunk(h);  // the graph holds the old descriptor
  XY_CUDA(cudaMemcpy(h->d_desc, &h->desc, sizeof(LatDesc), cudaMemcpyHostToDevice));
  return XY_OK;
}

xy_status xy_get_band_stats(xy_lattice *h, uint64_t *n_fp64, uint64_t *n_fp32_wrong) {
  if (!h) return fail(XY_EINVAL, "handle is NULL");
  XY_CUDA(cudaStreamSynchronize(h->stream));
  DevState s;
  XY_CUDA(cudaMemcpy(&s, h->d_state, sizeof(s), cudaMemcpyDeviceToHost));
  if (n_fp64) *n_fp64 = s.n_fp64;
  if (n_fp32_wrong) *n_fp32_wrong = s.n_fp32_wrong;
  return XY_OK;
}

// Checkpoint blob: header, device state, angles.
struct CkptHeader {
  char magic[8];
  uint32_t L, dtype, thr, tile_y;
  uint64_t seed;
  uint64_t enqueued;
  uint64_t state_bytes, angle_bytes;
};

xy_status xy_save(xy_lattice *h, void *host_blob, size_t *bytes) {
  if (!h || !bytes) return fail(XY_EINVAL, "NULL argument");
  const size_t ab = static_cast<size_t>(h->lo.L) * h->lo.L * h->lo.esize;
  const size_t need = sizeof(CkptHeader) + sizeof(DevState) + ab;
  if (!host_blob) {
    *bytes = need;
    return XY_OK;
  }
  if (*bytes < need) return fail(XY_ENOMEM, "blob of %zu bytes, %zu needed", *bytes, need);
  XY_CUDA(cudaStreamSynchronize(h->stream));
  char *p = static_cast<char *>(host_blob);
  CkptHeader hd;
  std::memcpy(hd.magic, "XYSWCK02", 8);
  hd.L = h->lo.L;
  hd.dtype = static_cast<uint32_t>(h->cfg.angle_dtype);
  hd.thr = static_cast<uint32_t>(h->cfg.threshold_mode);
  hd.tile_y = h->lo.TY;
  hd.seed = h->cfg.seed;
  hd.enqueued = h->enqueued;
  hd.state_bytes = sizeof(DevState);
  hd.angle_bytes = ab;
  std::memcpy(p, &hd, sizeof(hd));
  DevState s;
  XY_CUDA(cudaMemcpy(&s, h->d_state, sizeof(s), cudaMemcpyDeviceToHost));
  std::memcpy(p + sizeof(hd), &s, sizeof(s));
  XY_CUDA(cudaMemcpy(p + sizeof(hd) + sizeof(s), h->desc.theta[s.p[0].cur], ab,
                     cudaMemcpyDeviceToHost));
  *bytes = need;
  return XY_OK;
}

xy_status xy_load(xy_lattice *h, const void *host_blob, size_t bytes) {
  if (!h || !host_blob) return fail(XY_EINVAL, "NULL argument");
  const size_t ab = static_cast<size_t>(h->lo.L) * h->lo.L * h->lo.esize;
  if (bytes < sizeof(CkptHeader) + sizeof(DevState) + ab)
    return fail(XY_EINVAL, "blob too small");
  const char *p = static_cast<const char *>(host_blob);
  CkptHeader hd;
  std::memcpy(&hd, p, sizeof(hd));
  if (std::memcmp(hd.magic, "XYSWCK02", 8) != 0) return fail(XY_EINVAL, "not a checkpoint");
  if (hd.L != h->lo.L || hd.dtype != static_cast<uint32_t>(h->cfg.angle_dtype) ||
      hd.seed != h->cfg.seed || hd.state_bytes != sizeof(DevState) || hd.angle_bytes != ab)
    return fail(XY_EINVAL, "checkpoint does not match this lattice (L, dtype or seed)");
  DevState s;
  std::memcpy(&s, p + sizeof(hd), sizeof(s));
  XY_CUDA(cudaStreamSynchronize(h->stream));
  XY_CUDA(cudaMemcpy(h->desc.theta[s.p[0].cur], p + sizeof(hd) + sizeof(s), ab,
                     cudaMemcpyHostToDevice));
  XY_CUDA(cudaMemcpy(h->d_state, &s, sizeof(s), cudaMemcpyHostToDevice));
  XY_CUDA(cudaMemset(h->desc.acc, 0, sizeof(long long) * kSlots * kAccStride));
  h->enqueued = hd.enqueued;
  h->reported = hd.enqueued;
  return XY_OK;
}

}  // extern "C"
