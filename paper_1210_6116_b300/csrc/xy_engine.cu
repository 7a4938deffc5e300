// xy_engine.cu -- many independent lattices stepped by shared launches.
//
// An engine holds a table of active lattices (slots).  One sweep of all of
// them is the five kernels of a PCC sweep of a single lattice (k_finalize
// after every sweep: some lattices may run the PCC), each launched once for
// the whole table: the kernels walk a tile list spanning every lattice and
// find their lattice by a prefix search, so small lattices share the GPU
// instead of each paying its own launches.  The launches are captured in two
// CUDA graphs, of one sweep and of kEngineChunk sweeps; they are re-captured
// only when the active set changes (admission or retirement happens between
// sweeps).
//
// Every lattice keeps its own workspace, random numbers (seed, sweep
// counter), fixed-point observable sums and PCC state, so a lattice's results
// do not depend on which other lattices share the launches.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
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

xy_status fail(xy_status s, const char *fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  xy_set_last_error_message(msg);
  return s;
}

#define XY_CUDA(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      return fail(XY_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

struct Slot {
  bool active = false;
  xy_config cfg{};
  Layout lo{};
  LatDesc desc{};
  uint64_t enqueued = 0;
  uint64_t reported = 0;
};

template <int TY, typename AT, bool EXACT, bool FULL>
void launch_all(const LatDesc *descs, const uint32_t *prefix, uint32_t nrep, uint32_t nw,
                bool ext, cudaStream_t s) {
  launch_pdl(k_bond_label<TY, AT, EXACT, false, FULL>, nw, kThreads, bond_label_smem<TY>(), s, descs,
             prefix, nrep, nw, 0u, LatDesc{});
  const uint64_t items = static_cast<uint64_t>(nw) * (TY + 32);
  const uint64_t eb = (items + kThreads - 1) / kThreads;
  launch_pdl(k_merge<TY, FULL>, static_cast<uint32_t>(eb), kThreads, 0, s, descs, prefix, nrep, nw,
             LatDesc{});
  launch_pdl(k_compress<TY>, compress_blocks(nw), kThreads, 0, s, descs, prefix, nrep, nw,
             LatDesc{});
  // the engine exposes no labels: K4 never stores them (WL = false)
  if (ext)  // some lattice measures chik or runs Wolff; the others skip both by their flags
    launch_pdl(k_flip_measure<TY, AT, false, true, false, FULL>, nw, kThreads, flip_smem<TY>(), s, descs,
               prefix, nrep, nw, 0u, LatDesc{});
  else
    launch_pdl(k_flip_measure<TY, AT, false, false, false, FULL>, nw, kThreads, flip_smem<TY>(), s,
               descs, prefix, nrep, nw, 0u, LatDesc{});
  launch_pdl(k_finalize, nrep, kFinalizeThreads, 0, s, descs, nrep, 0u);
}

template <typename AT, bool EXACT, bool FULL>
void launch_ty_full(uint32_t TY, const LatDesc *descs, const uint32_t *prefix, uint32_t nrep,
                    uint32_t nw, bool ext, cudaStream_t s) {
  switch (TY) {
    case 16: launch_all<16, AT, EXACT, FULL>(descs, prefix, nrep, nw, ext, s); break;
    case 32: launch_all<32, AT, EXACT, FULL>(descs, prefix, nrep, nw, ext, s); break;
    case 64: launch_all<64, AT, EXACT, FULL>(descs, prefix, nrep, nw, ext, s); break;
    default: launch_all<128, AT, EXACT, FULL>(descs, prefix, nrep, nw, ext, s); break;
  }
}

// full: every lattice of the table is made of whole tiles (the FULL kernels)
template <typename AT, bool EXACT>
void launch_ty(uint32_t TY, const LatDesc *descs, const uint32_t *prefix, uint32_t nrep,
               uint32_t nw, bool ext, bool full, cudaStream_t s) {
  if (full) launch_ty_full<AT, EXACT, true>(TY, descs, prefix, nrep, nw, ext, s);
  else launch_ty_full<AT, EXACT, false>(TY, descs, prefix, nrep, nw, ext, s);
}

}  // namespace

struct xy_engine {
  uint32_t max_slots;
  int dtype, thr;
  uint32_t TY;
  cudaStream_t stream;     // the caller's stream: all work runs here
  cudaStream_t capture;    // private stream used only to record the graph
  LatDesc *d_descs;        // [max_slots], the active lattices, compacted
  uint32_t *d_prefix;      // [max_slots + 1], tile offsets of the table
  std::vector<Slot> slots;
  std::vector<LatDesc> h_descs;
  std::vector<uint32_t> h_prefix;
  std::vector<uint32_t> order;  // slot of table entry k
  uint32_t nrep = 0, nwork = 0;
  bool dirty = true;
  cudaGraphExec_t exec = nullptr;        // one sweep of every active lattice
  cudaGraphExec_t exec_chunk = nullptr;  // kEngineChunk such sweeps
};

namespace {

// Sweeps per replay of the engine's chunk graph.  A chunk keeps the
// programmatic-launch edges between its sweeps; one graph launch per sweep
// breaks that chain at every sweep.
constexpr uint32_t kEngineChunk = 4;

size_t table_bytes(uint32_t max_slots) {
  return align_up(sizeof(LatDesc) * max_slots, 256) + align_up(4u * (max_slots + 1u), 256);
}

void launch_table(xy_engine *e, cudaStream_t s) {
  bool ext = false, full = true;
  for (const LatDesc &d : e->h_descs) {
    ext = ext || d.xi || d.wolff;
    full = full && d.L % 32u == 0u && d.L % e->TY == 0u;
  }
  const bool ex = e->thr == XY_THR_F64;
  if (e->dtype == XY_F32) {
    if (ex) launch_ty<float, true>(e->TY, e->d_descs, e->d_prefix, e->nrep, e->nwork, ext, full, s);
    else launch_ty<float, false>(e->TY, e->d_descs, e->d_prefix, e->nrep, e->nwork, ext, full, s);
  } else if (e->dtype == XY_F16) {
    if (ex) launch_ty<__half, true>(e->TY, e->d_descs, e->d_prefix, e->nrep, e->nwork, ext, full, s);
    else launch_ty<__half, false>(e->TY, e->d_descs, e->d_prefix, e->nrep, e->nwork, ext, full, s);
  } else {
    if (ex) launch_ty<uint16_t, true>(e->TY, e->d_descs, e->d_prefix, e->nrep, e->nwork, ext, full, s);
    else launch_ty<uint16_t, false>(e->TY, e->d_descs, e->d_prefix, e->nrep, e->nwork, ext, full, s);
  }
}

// Upload the compacted table of active lattices and record the graph of one
// sweep over it.
xy_status rebuild(xy_engine *e) {
  XY_CUDA(cudaStreamSynchronize(e->stream));  // host table buffers are reused
  e->order.clear();
  e->h_descs.clear();
  e->h_prefix.assign(1, 0u);
  for (uint32_t k = 0; k < e->max_slots; ++k) {
    if (!e->slots[k].active) continue;
    e->order.push_back(k);
    e->h_descs.push_back(e->slots[k].desc);
    e->h_prefix.push_back(e->h_prefix.back() + e->slots[k].lo.ntiles);
  }
  e->nrep = static_cast<uint32_t>(e->order.size());
  e->nwork = e->h_prefix.back();
  for (cudaGraphExec_t *g : {&e->exec, &e->exec_chunk}) {
    if (*g) cudaGraphExecDestroy(*g);
    *g = nullptr;
  }
  e->dirty = false;
  if (e->nrep == 0) return XY_OK;
  XY_CUDA(cudaMemcpyAsync(e->d_descs, e->h_descs.data(), sizeof(LatDesc) * e->nrep,
                          cudaMemcpyHostToDevice, e->stream));
  XY_CUDA(cudaMemcpyAsync(e->d_prefix, e->h_prefix.data(), 4u * (e->nrep + 1u),
                          cudaMemcpyHostToDevice, e->stream));
  XY_CUDA(cudaStreamSynchronize(e->stream));
  for (uint32_t sweeps : {1u, kEngineChunk}) {
    cudaGraph_t graph = nullptr;
    XY_CUDA(cudaStreamBeginCapture(e->capture, cudaStreamCaptureModeThreadLocal));
    for (uint32_t k = 0; k < sweeps; ++k) launch_table(e, e->capture);
    cudaError_t le = cudaGetLastError();
    cudaError_t ce = cudaStreamEndCapture(e->capture, &graph);
    if (le != cudaSuccess || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return fail(XY_ECUDA, "graph capture: %s", cudaGetErrorString(le != cudaSuccess ? le : ce));
    }
    cudaError_t ie = cudaGraphInstantiate(sweeps == 1u ? &e->exec : &e->exec_chunk, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return fail(XY_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
  }
  return XY_OK;
}

}  // namespace

extern "C" {

xy_status xy_engine_workspace_size(uint32_t max_slots, size_t *bytes) {
  if (!bytes || max_slots == 0) return fail(XY_EINVAL, "max_slots must be >= 1");
  *bytes = table_bytes(max_slots);
  return XY_OK;
}

xy_status xy_engine_create(uint32_t max_slots, int angle_dtype, int threshold_mode,
                           uint32_t tile_y, void *d_workspace, size_t bytes, void *cuda_stream,
                           xy_engine **out) {
  if (!out) return fail(XY_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_slots == 0) return fail(XY_EINVAL, "max_slots must be >= 1");
  if (angle_dtype != XY_F32 && angle_dtype != XY_F16 && angle_dtype != XY_U16)
    return fail(XY_EINVAL, "bad angle_dtype");
  if (threshold_mode != XY_THR_F32 && threshold_mode != XY_THR_F64)
    return fail(XY_EINVAL, "bad threshold_mode");
  if (!tile_ok(tile_y)) return fail(XY_EINVAL, "tile_y must be 16, 32, 64 or 128");
  if (!d_workspace || reinterpret_cast<uintptr_t>(d_workspace) % 256)
    return fail(XY_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (bytes < table_bytes(max_slots)) return fail(XY_ENOMEM, "engine workspace too small");
  xy_engine *e = new (std::nothrow) xy_engine();
  if (!e) return fail(XY_ENOMEM, "host allocation failed");
  e->max_slots = max_slots;
  e->dtype = angle_dtype;
  e->thr = threshold_mode;
  e->TY = tile_y;
  e->stream = static_cast<cudaStream_t>(cuda_stream);
  char *ws = static_cast<char *>(d_workspace);
  e->d_descs = reinterpret_cast<LatDesc *>(ws);
  e->d_prefix = reinterpret_cast<uint32_t *>(ws + align_up(sizeof(LatDesc) * max_slots, 256));
  e->slots.resize(max_slots);
  cudaError_t ce = cudaStreamCreateWithFlags(&e->capture, cudaStreamNonBlocking);
  if (ce != cudaSuccess) {
    delete e;
    return fail(XY_ECUDA, "capture stream: %s", cudaGetErrorString(ce));
  }
  *out = e;
  return XY_OK;
}

xy_status xy_engine_admit(xy_engine *e, const xy_config *cfg, const xy_pcc_params *pcc,
                          void *d_workspace, size_t bytes, uint32_t *slot) {
  if (!e || !cfg || !slot) return fail(XY_EINVAL, "NULL argument");
  xy_config c = *cfg;
  c.tile_y = e->TY;
  Layout lo;
  xy_status st = make_layout(&c, &lo);
  if (st != XY_OK) return st;
  if (c.angle_dtype != e->dtype || c.threshold_mode != e->thr)
    return fail(XY_EINVAL, "angle_dtype / threshold_mode differ from the engine's");
  if (c.L % 32 != 0) return fail(XY_EUNSUPPORTED, "engine lattices need L divisible by 32");
  if (!d_workspace || reinterpret_cast<uintptr_t>(d_workspace) % 256)
    return fail(XY_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (bytes < lo.total) return fail(XY_ENOMEM, "workspace of %zu bytes, %zu needed", bytes, lo.total);
  if (pcc && (pcc->block == 0 || !(pcc->dbeta0 >= 0.0)))
    return fail(XY_EINVAL, "PCC block must be >= 1 and dbeta0 >= 0");
  uint32_t k = 0;
  while (k < e->max_slots && e->slots[k].active) ++k;
  if (k == e->max_slots) return fail(XY_ENOMEM, "all %u slots are in use", e->max_slots);
  Slot &s = e->slots[k];
  s = Slot();
  s.cfg = c;
  s.lo = lo;
  s.desc = make_desc(&c, lo, static_cast<char *>(d_workspace));
  XY_CUDA(cudaMemsetAsync(s.desc.acc, 0, sizeof(long long) * kSlots * kAccStride, e->stream));
  XY_CUDA(cudaMemsetAsync(s.desc.coin, 0, (static_cast<size_t>(lo.L) * lo.L / 32 + 2) * 4, e->stream));
  k_init_state<<<1, 1, 0, e->stream>>>(s.desc, c.beta, c.angle_dtype == XY_U16 ? 1u : 0u);
  k_init_wave<<<(lo.L + 255) / 256, 256, 0, e->stream>>>(s.desc);
  const uint64_t n = static_cast<uint64_t>(lo.L) * lo.L;
  const uint32_t blocks = static_cast<uint32_t>(std::min<uint64_t>((n + 255) / 256, 4096));
  if (c.angle_dtype == XY_F32)
    k_init_angles<float><<<blocks, 256, 0, e->stream>>>(s.desc, c.start);
  else if (c.angle_dtype == XY_F16)
    k_init_angles<__half><<<blocks, 256, 0, e->stream>>>(s.desc, c.start);
  else
    k_init_angles<uint16_t><<<blocks, 256, 0, e->stream>>>(s.desc, c.start);
  if (pcc)
    k_set_pcc<<<1, 1, 0, e->stream>>>(s.desc.st, 1u, pcc->target, pcc->dbeta0, pcc->halve_every,
                                      pcc->block);
  XY_CUDA(cudaGetLastError());
  s.active = true;
  e->dirty = true;
  *slot = k;
  return XY_OK;
}

xy_status xy_engine_retire(xy_engine *e, uint32_t slot) {
  if (!e || slot >= e->max_slots || !e->slots[slot].active)
    return fail(XY_EINVAL, "no active lattice in that slot");
  XY_CUDA(cudaStreamSynchronize(e->stream));
  e->slots[slot].active = false;
  e->dirty = true;
  return XY_OK;
}

xy_status xy_engine_step(xy_engine *e, uint32_t n_sweeps) {
  if (!e) return fail(XY_EINVAL, "engine is NULL");
  if (e->dirty) {
    xy_status s = rebuild(e);
    if (s != XY_OK) return s;
  }
  if (e->nrep == 0 || n_sweeps == 0) return XY_OK;
  nvtxRangePushA("xy_engine_step");
  for (uint32_t k = 0; k < n_sweeps;) {
    const bool chunk = n_sweeps - k >= kEngineChunk;
    const cudaError_t ge = cudaGraphLaunch(chunk ? e->exec_chunk : e->exec, e->stream);
    if (ge != cudaSuccess) {
      nvtxRangePop();
      return fail(XY_ECUDA, "cudaGraphLaunch failed: %s", cudaGetErrorString(ge));
    }
    k += chunk ? kEngineChunk : 1u;
  }
  nvtxRangePop();
  for (uint32_t k : e->order) e->slots[k].enqueued += n_sweeps;
  return XY_OK;
}

xy_status xy_engine_measure(xy_engine *e, uint32_t slot, xy_obs *out, uint32_t max_records,
                            uint32_t *n_out) {
  if (!e || !n_out || slot >= e->max_slots || !e->slots[slot].active)
    return fail(XY_EINVAL, "bad engine, slot or n_out");
  if (max_records && !out) return fail(XY_EINVAL, "out is NULL");
  Slot &s = e->slots[slot];
  XY_CUDA(cudaStreamSynchronize(e->stream));
  uint32_t err = 0;
  XY_CUDA(cudaMemcpy(&err, &s.desc.st->err, sizeof(err), cudaMemcpyDeviceToHost));
  if (err) {
    XY_CUDA(cudaMemset(&s.desc.st->err, 0, sizeof(err)));  // reported once
    return device_error_status(err);
  }
  const uint64_t pending = s.enqueued - s.reported;
  const uint64_t take = std::min<uint64_t>(std::min<uint64_t>(pending, s.lo.rec_cap), max_records);
  const uint64_t first = s.enqueued - take;
  for (uint64_t k = 0; k < take;) {
    const uint64_t pos = (first + k) % s.lo.rec_cap;
    const uint64_t run = std::min<uint64_t>(take - k, s.lo.rec_cap - pos);
    XY_CUDA(cudaMemcpy(out + k, s.desc.rec + pos, run * sizeof(xy_obs), cudaMemcpyDeviceToHost));
    k += run;
  }
  s.reported = s.enqueued;
  *n_out = static_cast<uint32_t>(take);
  return XY_OK;
}

xy_status xy_engine_get_angles(xy_engine *e, uint32_t slot, void *host_dst) {
  if (!e || !host_dst || slot >= e->max_slots || !e->slots[slot].active)
    return fail(XY_EINVAL, "bad engine, slot or buffer");
  Slot &s = e->slots[slot];
  XY_CUDA(cudaStreamSynchronize(e->stream));
  DevState st;
  XY_CUDA(cudaMemcpy(&st, s.desc.st, sizeof(st), cudaMemcpyDeviceToHost));
  XY_CUDA(cudaMemcpy(host_dst, s.desc.theta[st.p[0].cur],
                     static_cast<size_t>(s.lo.L) * s.lo.L * s.lo.esize, cudaMemcpyDeviceToHost));
  return XY_OK;
}

xy_status xy_engine_get_state(xy_engine *e, uint32_t slot, double *beta, uint64_t *sweep) {
  if (!e || slot >= e->max_slots || !e->slots[slot].active)
    return fail(XY_EINVAL, "bad engine or slot");
  XY_CUDA(cudaStreamSynchronize(e->stream));
  DevState st;
  XY_CUDA(cudaMemcpy(&st, e->slots[slot].desc.st, sizeof(st), cudaMemcpyDeviceToHost));
  if (beta) *beta = st.p[0].beta;
  if (sweep) *sweep = st.p[0].t;
  return XY_OK;
}

xy_status xy_engine_destroy(xy_engine *e) {
  if (!e) return fail(XY_EINVAL, "engine is NULL");
  cudaStreamSynchronize(e->stream);
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->exec_chunk) cudaGraphExecDestroy(e->exec_chunk);
  cudaStreamDestroy(e->capture);
  delete e;
  return XY_OK;
}

}  // extern "C"
