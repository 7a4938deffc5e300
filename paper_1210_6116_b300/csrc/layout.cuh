// layout.cuh -- workspace layout of one lattice and its device descriptor,
// shared by the single-lattice API (xy_api.cu) and the engine (xy_engine.cu).
#pragma once

#include <cmath>
#include <cstdint>
#include <cstdio>

#include "../../include/xy.h"
#include "sweep_kernels.cuh"

// Sets the calling thread's xy_last_error() message (defined in xy_api.cu).
void xy_set_last_error_message(const char *msg);

namespace xyk {

inline xy_status layout_fail(xy_status s, const char *msg) {
  xy_set_last_error_message(msg);
  return s;
}

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Status for a lattice's device error word (DevState::err): a bounded
// find / union / jump loop that ran out is XY_ETIMEOUT, any other recorded
// error XY_EINTERNAL.  Every entry point that reports device errors maps the
// word through here, so they agree.
inline xy_status device_error_status(uint32_t err) {
  char msg[128];
  if (err & (kErrFindCap | kErrUnionCap)) {
    snprintf(msg, sizeof(msg), "device-side find/union loop hit its bound (err=%#x)", err);
    return layout_fail(XY_ETIMEOUT, msg);
  }
  if (err) {
    snprintf(msg, sizeof(msg), "device error word %#x", err);
    return layout_fail(XY_EINTERNAL, msg);
  }
  return XY_OK;
}

inline uint32_t default_tile_y(uint32_t L) {
  if (L <= 32) return 16;
  if (L <= 256) return 32;
  return 64;
}

inline bool tile_ok(uint32_t ty) { return ty == 16 || ty == 32 || ty == 64 || ty == 128; }

struct Layout {
  uint32_t L, TY, ntx, nty, ntiles, rec_cap;
  size_t esize;
  size_t off_state, off_desc, off_prefix, off_acc, off_rec, off_theta0,
      off_theta1, off_label, off_rplane, off_dplane, off_edge, off_links, off_link_count, off_coin,
      off_wave, total;
};

inline xy_status make_layout(const xy_config *c, Layout *lo) {
  if (!c) return layout_fail(XY_EINVAL, "config is NULL");
  if (c->L < 2 || c->L > 65536)
    return layout_fail(XY_EINVAL, "L outside 2..65536");
  if (!(c->beta >= 0.0) || !std::isfinite(c->beta))
    return layout_fail(XY_EINVAL, "beta must be finite and >= 0");
  if (c->angle_dtype != XY_F32 && c->angle_dtype != XY_F16 && c->angle_dtype != XY_U16)
    return layout_fail(XY_EINVAL, "angle_dtype must be XY_F32, XY_F16 or XY_U16");
  if (c->threshold_mode != XY_THR_F32 && c->threshold_mode != XY_THR_F64)
    return layout_fail(XY_EINVAL, "threshold_mode must be XY_THR_F32 or XY_THR_F64");
  if (c->start != 0 && c->start != 1)
    return layout_fail(XY_EINVAL, "start must be 0 (random) or 1 (ordered)");
  if (c->measure_xi > 1 || c->update > XY_UPDATE_WOLFF)
    return layout_fail(XY_EINVAL, "measure_xi must be 0 or 1, update XY_UPDATE_SW or XY_UPDATE_WOLFF");
  const uint32_t ty = c->tile_y ? c->tile_y : default_tile_y(c->L);
  if (!tile_ok(ty)) return layout_fail(XY_EINVAL, "tile_y must be 16, 32, 64 or 128");
  lo->L = c->L;
  lo->TY = ty;
  lo->ntx = (c->L + 31) / 32;
  lo->nty = (c->L + ty - 1) / ty;
  lo->ntiles = lo->ntx * lo->nty;
  lo->rec_cap = c->record_cap ? c->record_cap : 4096;
  lo->esize = c->angle_dtype == XY_F32 ? 4 : 2;
  const uint64_t n = static_cast<uint64_t>(c->L) * c->L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  lo->off_state = take(sizeof(DevState));
  lo->off_desc = take(sizeof(LatDesc));
  lo->off_prefix = take(2 * sizeof(uint32_t));
  lo->off_acc = take(sizeof(long long) * kSlots * kAccStride);
  lo->off_rec = take(sizeof(ObsRecord) * lo->rec_cap);
  lo->off_theta0 = take(n * lo->esize);
  lo->off_theta1 = take(n * lo->esize);
  lo->off_label = take(n * sizeof(uint32_t));
  lo->off_rplane = take(static_cast<size_t>(lo->ntiles) * ty * sizeof(uint32_t));
  lo->off_dplane = take(static_cast<size_t>(lo->ntiles) * ty * sizeof(uint32_t));
  lo->off_edge = take(static_cast<size_t>(lo->ntiles) * (2 * ty + 64) * sizeof(uint32_t));
  lo->off_links = take(static_cast<size_t>(lo->ntiles) * (ty + 32) * sizeof(uint32_t));
  lo->off_link_count = take(static_cast<size_t>(lo->ntiles) * sizeof(uint32_t));
  lo->off_coin = take((n / 32 + 2) * sizeof(uint32_t));
  lo->off_wave = take(static_cast<size_t>(c->L) * 8);
  lo->total = off;
  return XY_OK;
}


// Device descriptor of a lattice whose workspace starts at ws.
inline LatDesc make_desc(const xy_config *cfg, const Layout &lo, char *ws) {
  LatDesc d{};
  d.L = lo.L;
  d.ntx = lo.ntx;
  d.nty = lo.nty;
  d.ntiles = lo.ntiles;
  d.key0 = static_cast<uint32_t>(cfg->seed & 0xFFFFFFFFu);
  d.key1 = static_cast<uint32_t>(cfg->seed >> 32);
  d.rec_cap = lo.rec_cap;
  d.ragged = (lo.L % 32) != 0;
  d.Lmagic = ~0ull / lo.L + 1ull;
  d.ntx_magic = ~0ull / lo.ntx + 1ull;
  d.inv_n = 1.0 / (static_cast<double>(lo.L) * lo.L);
  d.theta[0] = ws + lo.off_theta0;
  d.theta[1] = ws + lo.off_theta1;
  d.label = reinterpret_cast<uint32_t *>(ws + lo.off_label);
  d.rplane = reinterpret_cast<uint32_t *>(ws + lo.off_rplane);
  d.dplane = reinterpret_cast<uint32_t *>(ws + lo.off_dplane);
  d.edge = reinterpret_cast<uint32_t *>(ws + lo.off_edge);
  d.links = reinterpret_cast<uint32_t *>(ws + lo.off_links);
  d.link_count = reinterpret_cast<uint32_t *>(ws + lo.off_link_count);
  d.coin = reinterpret_cast<uint32_t *>(ws + lo.off_coin);
  d.xi = cfg->measure_xi ? 1u : 0u;
  d.wolff = cfg->update == XY_UPDATE_WOLFF ? 1u : 0u;
  d.wave = reinterpret_cast<const float2 *>(ws + lo.off_wave);
  d.find_cap = kFindCap;
  d.link_cap = lo.TY + 32u;
  d.acc = reinterpret_cast<long long *>(ws + lo.off_acc);
  d.st = reinterpret_cast<DevState *>(ws + lo.off_state);
  d.rec = reinterpret_cast<ObsRecord *>(ws + lo.off_rec);
  return d;
}

}  // namespace xyk
