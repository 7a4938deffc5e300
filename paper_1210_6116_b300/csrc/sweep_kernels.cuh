// sweep_kernels.cuh -- the sm_103a kernels of one Swendsen-Wang sweep of the
// 2D XY model in Wolff's embedding (Komura & Okabe, Secs. 1-2; Eq. (3)).
//
// Per sweep t, on every lattice of a launch (one lattice, or a batch of
// independent replicas that share the launch):
//   k_bond_label   projection a_i = s_i.r, right/down bonds with
//                  p = 1 - exp(-2 beta a_i a_j), 2-bit masks (two bit planes),
//                  cluster coin bits, then union-find inside the 32 x TY tile
//                  in shared memory; writes tile-local labels (global index of
//                  the tile-local minimum site).
//   k_merge        union of the tile-local clusters across tile edges in the
//                  global label array (CAS linking, smaller index wins, so the
//                  final root is the minimum site index of the cluster).
//   k_compress     points every merged tile root straight at its final root.
//   k_flip_measure canonical label of every site, Wolff reflection
//                  theta' = C - theta (mod 2 pi) of clusters whose root coin is
//                  1, and the observable sums of Eqs. (3)-(6) on the new
//                  configuration, in exact integer fixed point.
//   k_finalize     FP64 observables, the record ring, the helicity-modulus PCC
//                  step (Sec. 2) and the random axis of the next sweep.
//
// Layouts (per lattice, N = L*L, i = y*L + x):
//   theta[2]  angle double buffer (FP32 or FP16); the sweep reads theta[cur]
//             and writes theta[cur ^ 1], so halo reads never race with flips.
//   label     N uint32.
//   rplane,   tile-major bond bit planes: word (tile*TY + r) holds the right
//   dplane    (down) bonds of tile row r, bit c = column x0 + c.
//   coin      linear bit array, bit i = coin of site i (read only for roots).
//   acc       kSlots x 8 int64 accumulators of the fixed-point sums.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

#include "philox.cuh"

namespace xyk {

constexpr int kThreads = 256;          // 8 warps per tile CTA
constexpr int kWarps = kThreads / 32;
constexpr int kSlots = 64;             // accumulator slots per lattice
constexpr int kAccStride = 8;          // int64 per slot (6 used)
constexpr uint32_t kFindCap = 1u << 22;  // bound on any global find / union loop

// error bits recorded in DevState::err
constexpr uint32_t kErrFindCap = 1u;
constexpr uint32_t kErrUnionCap = 2u;

// Fixed-point scale of the observable sums: each FP32 term in [-1, 1] is
// rounded to a multiple of 2^-22 and summed exactly in integers.
constexpr double kFixScale = 4194304.0;  // 2^22

struct ObsRecord {  // identical layout to xy_obs
  double energy_per_site, m2, mx, my, ex, sx, ey, sy, upsilon, beta;
  uint64_t sweep;
};

struct DevState {
  // parameters of the next sweep
  uint32_t t;      // sweep counter
  uint32_t cur;    // theta buffer holding the current angles
  double beta;
  double cphi, sphi;     // axis of sweep t (FP64)
  float cphi32, sphi32;  // FP32 copies
  float c32;             // reflection constant: theta' = c32 - theta (mod 2pi)
  float beta2_32;        // 2 beta in FP32
  float eps;             // half-width of the FP32 error band of exact mode
  uint32_t pcc_on;
  // helicity-modulus PCC
  uint32_t pcc_block, pcc_halve, pcc_count, pad1;
  double pcc_target, pcc_dbeta0, pcc_acc;
  uint64_t pcc_k;
  // records
  uint64_t rec_count;
  // diagnostics
  unsigned long long n_fp64, n_fp32_wrong;
  uint32_t err, pad2;
};

struct LatDesc {
  uint32_t L, ntx, nty, ntiles;
  uint32_t key0, key1, rec_cap, ragged;
  void *theta[2];
  uint32_t *label;
  uint32_t *rplane, *dplane;
  uint32_t *coin;
  long long *acc;
  DevState *st;
  ObsRecord *rec;
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float two_pi_f() { return 6.2831854820251465f; }
__device__ __forceinline__ float pi_f() { return 3.14159274101257324f; }

template <typename AT>
__device__ __forceinline__ float load_angle(const AT *p, uint64_t i);
template <>
__device__ __forceinline__ float load_angle<float>(const float *p, uint64_t i) {
  return __ldg(p + i);
}
template <>
__device__ __forceinline__ float load_angle<__half>(const __half *p,
                                                    uint64_t i) {
  return __half2float(__ldg(p + i));
}

// wrap an FP32 angle in (-2pi, 2pi] into [0, 2pi) with FP32 adds
__device__ __forceinline__ float wrap_angle(float v) {
  if (v < 0.0f) v = __fadd_rn(v, two_pi_f());
  if (v >= two_pi_f()) v = __fadd_rn(v, -two_pi_f());
  return v;
}

template <typename AT>
__device__ __forceinline__ AT store_value(float v);
template <>
__device__ __forceinline__ float store_value<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ __half store_value<__half>(float v) {
  __half h = __float2half_rn(v);
  const float back = __half2float(h);
  if (back >= two_pi_f()) h = __float2half_rn(__fadd_rn(back, -two_pi_f()));
  return h;
}
template <typename AT>
__device__ __forceinline__ float stored_float(AT v);
template <>
__device__ __forceinline__ float stored_float<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ float stored_float<__half>(__half v) {
  return __half2float(v);
}

// projection s.r in FP32 from the stored angle; sin/cos through the SFU on
// the centred argument theta - pi_f in [-pi, pi)
__device__ __forceinline__ float project32(float th, float cphi, float sphi) {
  float s, c;
  __sincosf(__fadd_rn(th, -pi_f()), &s, &c);  // s = -sin th, c = -cos th
  return -fmaf(c, cphi, s * sphi);
}

// FP64 projection exactly as the rule defines it: cos(th) cphi + sin(th) sphi
__device__ __forceinline__ double project64(float th, double cphi,
                                            double sphi) {
  double s, c;
  sincos(static_cast<double>(th), &s, &c);
  return __dadd_rn(__dmul_rn(c, cphi), __dmul_rn(s, sphi));
}

__device__ __forceinline__ uint32_t find_rep(const uint32_t *__restrict__ pre,
                                             uint32_t nrep, uint32_t work) {
  uint32_t lo = 0, hi = nrep;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(pre + mid) <= work) lo = mid;
    else hi = mid;
  }
  return lo;
}

struct Tile {
  uint32_t x0, y0, w, h, xh, yh;
};

template <int TY>
__device__ __forceinline__ Tile tile_geom(uint32_t L, uint32_t ntx,
                                          uint32_t tile) {
  Tile g;
  const uint32_t tx = tile % ntx, ty = tile / ntx;
  g.x0 = tx * 32u;
  g.y0 = ty * static_cast<uint32_t>(TY);
  g.w = min(32u, L - g.x0);
  g.h = min(static_cast<uint32_t>(TY), L - g.y0);
  g.xh = (g.x0 + g.w == L) ? 0u : g.x0 + g.w;  // column right of the tile
  g.yh = (g.y0 + g.h == L) ? 0u : g.y0 + g.h;  // row below the tile
  return g;
}

// ---------------------------------------------------------------------------
// bond decision
// ---------------------------------------------------------------------------
// FP64 rule, operation for operation: x = a_i a_j; active iff x > 0 and
// (w + 1/2) 2^-32 < 1 - exp(-2 beta x).
static __device__ __noinline__ bool bond_fp64(float th_i, float th_j, uint32_t word,
                                       double beta, double cphi, double sphi) {
  const double ai = project64(th_i, cphi, sphi);
  const double aj = project64(th_j, cphi, sphi);
  const double x = __dmul_rn(ai, aj);
  if (!(x > 0.0)) return false;
  const double p = __dsub_rn(1.0, exp(__dmul_rn(__dmul_rn(-2.0, beta), x)));
  const double u = __dmul_rn(__dadd_rn(static_cast<double>(word), 0.5),
                             0x1p-32);
  return u < p;
}

// ---------------------------------------------------------------------------
// shared-memory union-find on tile-local indices (r*32 + c).  Every link
// points to a strictly smaller index, so finds terminate.  Finds halve the
// path: a node is re-pointed at its grandparent, which is always an ancestor,
// so concurrent halving and CAS linking of roots never lose a union.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t sfind(volatile uint32_t *par, uint32_t a) {
  uint32_t p = par[a];
  while (p != a) {
    const uint32_t gp = par[p];
    if (gp != p) par[a] = gp;
    a = gp;
    p = par[a];
  }
  return a;
}

__device__ __forceinline__ void sunion(uint32_t *par, uint32_t a, uint32_t b) {
  volatile uint32_t *vp = par;
  a = sfind(vp, a);
  b = sfind(vp, b);
  while (a != b) {
    if (a < b) {
      const uint32_t tmp = a;
      a = b;
      b = tmp;
    }
    const uint32_t old = atomicCAS(par + a, a, b);  // link root a under b
    if (old == a) return;
    a = sfind(vp, old);
    b = sfind(vp, b);
  }
}

// ---------------------------------------------------------------------------
// global union-find on site indices (label array)
// ---------------------------------------------------------------------------
// find with path halving; only used while no other kernel reads labels
__device__ __forceinline__ uint32_t gfind_halve(uint32_t *lab, uint32_t a,
                                                DevState *st) {
  for (uint32_t it = 0; it < kFindCap; ++it) {
    const uint32_t p = __ldcg(lab + a);
    if (p == a) return a;
    const uint32_t gp = __ldcg(lab + p);
    if (gp != p) __stcg(lab + a, gp);  // gp is an ancestor: safe to skip p
    a = gp;
  }
  atomicOr(&st->err, kErrFindCap);
  return a;
}

// read-only find
__device__ __forceinline__ uint32_t gfind_ro(const uint32_t *lab, uint32_t a,
                                             DevState *st) {
  for (uint32_t it = 0; it < kFindCap; ++it) {
    const uint32_t p = __ldcg(lab + a);
    if (p == a) return a;
    a = p;
  }
  atomicOr(&st->err, kErrFindCap);
  return a;
}

__device__ __forceinline__ void gunion(uint32_t *lab, uint32_t a, uint32_t b,
                                       DevState *st) {
  a = gfind_halve(lab, a, st);
  b = gfind_halve(lab, b, st);
  for (uint32_t it = 0; a != b; ++it) {
    if (it >= kFindCap) {
      atomicOr(&st->err, kErrUnionCap);
      return;
    }
    if (a < b) {
      const uint32_t tmp = a;
      a = b;
      b = tmp;
    }
    const uint32_t old = atomicCAS(lab + a, a, b);
    if (old == a) return;
    a = gfind_halve(lab, old, st);
    b = gfind_halve(lab, b, st);
  }
}

// ---------------------------------------------------------------------------
// Tile union-find over bond words already in shared memory (sR, sD).
// Row runs come from the right-bond word by bit scans; vertical unions are
// issued only at the first column of each pair of vertically touching runs.
// Writes tile-local labels (global index of the tile minimum) to `label`.
// ---------------------------------------------------------------------------
template <int TY>
__device__ __forceinline__ void tile_label(const Tile &g, uint32_t L,
                                           const uint32_t *sR,
                                           const uint32_t *sD, uint32_t *par,
                                           uint32_t *label) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rmask = (g.w >= 32u) ? 0x7FFFFFFFu : ((1u << (g.w - 1u)) - 1u);
  const bool col_ok = lane < static_cast<int>(g.w);
  // every site points at the start of its row run; run starts are roots
  for (uint32_t r = warp; r < g.h; r += kWarps) {
    if (col_ok) {
      const uint32_t starts = ~((sR[r] & rmask) << 1);
      const uint32_t s = 31u - __clz(starts & (0xFFFFFFFFu >> (31 - lane)));
      par[r * 32u + lane] = r * 32u + s;
    }
  }
  __syncthreads();
  // Vertical unions, merged hierarchically: at span s, row blocks
  // [2ks, 2ks + s) and [2ks + s, 2ks + 2s) join across their boundary row
  // pair only.  Boundaries of one level touch disjoint node sets, and a
  // node is at most one link per level from its block root, so trees stay
  // log2(TY) deep.  One union per pair of vertically touching runs (the
  // first column where they touch).
  for (uint32_t span = 1; span < g.h; span <<= 1) {
    const uint32_t nb = (g.h - span + 2u * span - 1u) / (2u * span);
    for (uint32_t b = warp; b < nb; b += kWarps) {
      const uint32_t r = b * 2u * span + span - 1u;
      if (r + 1u < g.h) {
        const uint32_t D = sD[r];
        const uint32_t V = D & ~((D & sR[r] & sR[r + 1] & rmask) << 1);
        if (col_ok && ((V >> lane) & 1u))
          sunion(par, r * 32u + lane, (r + 1u) * 32u + lane);
      }
    }
    __syncthreads();
  }
  // run starts point straight at their root; every other site is then two
  // hops from it (all ancestors of a site are run starts)
  for (uint32_t r = warp; r < g.h; r += kWarps) {
    const uint32_t starts = ~((sR[r] & rmask) << 1);
    if (col_ok && ((starts >> lane) & 1u)) {
      const uint32_t node = r * 32u + lane;
      par[node] = sfind(par, node);
    }
  }
  __syncthreads();
  for (uint32_t r = warp; r < g.h; r += kWarps) {
    if (col_ok) {
      const uint32_t root = par[par[r * 32u + lane]];
      label[static_cast<uint64_t>(g.y0 + r) * L + g.x0 + lane] =
          (g.y0 + (root >> 5)) * L + g.x0 + (root & 31u);
    }
  }
}

template <int TY>
constexpr size_t bond_label_smem() {
  return sizeof(float) * (TY + 1) * 33 + sizeof(uint32_t) * (TY * 32 + 2 * TY);
}

// ---------------------------------------------------------------------------
// K1: projection + bonds + coins + tile labels
// ---------------------------------------------------------------------------
template <int TY, typename AT, bool EXACT, bool FROM_PLANES>
__global__ void __launch_bounds__(kThreads)
    k_bond_label(const LatDesc *__restrict__ descs,
                 const uint32_t *__restrict__ prefix, uint32_t nrep,
                 uint32_t nwork) {
  extern __shared__ __align__(16) unsigned char smem[];
  float(*sa)[33] = reinterpret_cast<float(*)[33]>(smem);
  uint32_t *par =
      reinterpret_cast<uint32_t *>(smem + sizeof(float) * (TY + 1) * 33);
  uint32_t *sR = par + TY * 32;
  uint32_t *sD = sR + TY;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (uint32_t work = blockIdx.x; work < nwork; work += gridDim.x) {
    const uint32_t rep = find_rep(prefix, nrep, work);
    const LatDesc &d = descs[rep];
    const uint32_t tile = work - __ldg(prefix + rep);
    const uint32_t L = d.L;
    const Tile g = tile_geom<TY>(L, d.ntx, tile);
    DevState *st = d.st;

    if (!FROM_PLANES) {
      const uint32_t t = st->t;
      const AT *th = static_cast<const AT *>(d.theta[st->cur]);
      const float cphi = st->cphi32, sphi = st->sphi32;
      // projections of the tile plus its right column and bottom row; all
      // loads of a thread are issued before the first use
      // (thread t < h also loads row t of the column right of the tile)
      constexpr int KR = TY / kWarps + 1;
      float tv[KR];
#pragma unroll
      for (int k = 0; k < KR; ++k) {
        const uint32_t r = warp + k * kWarps;
        tv[k] = 0.0f;
        if (r <= g.h && lane < static_cast<int>(g.w)) {
          const uint64_t row = static_cast<uint64_t>(r < g.h ? g.y0 + r : g.yh) * L;
          tv[k] = load_angle(th, row + g.x0 + lane);
        }
      }
      const bool hc = threadIdx.x < g.h;
      float thc = 0.0f;
      if (hc) thc = load_angle(th, static_cast<uint64_t>(g.y0 + threadIdx.x) * L + g.xh);
#pragma unroll
      for (int k = 0; k < KR; ++k) {
        const uint32_t r = warp + k * kWarps;
        if (r <= g.h && lane < static_cast<int>(g.w)) sa[r][lane] = project32(tv[k], cphi, sphi);
      }
      if (hc) sa[threadIdx.x][g.w] = project32(thc, cphi, sphi);
      __syncthreads();
      const float b2 = st->beta2_32, eps = st->eps;
      for (uint32_t r = warp; r < g.h; r += kWarps) {
        const uint32_t gy = g.y0 + r;
        bool br = false, bd = false, cn = false;
        if (lane < static_cast<int>(g.w)) {
          const uint32_t i = gy * L + g.x0 + lane;
          const Words4 rn = philox4x32_10(i, 0u, t, kDomBond, d.key0, d.key1);
          const float ai = sa[r][lane];
          const float u0 = fmaf(static_cast<float>(rn.w0), 0x1p-32f, 0x1p-33f);
          const float u1 = fmaf(static_cast<float>(rn.w1), 0x1p-32f, 0x1p-33f);
          const float xr = ai * sa[r][lane + 1];
          const float xd = ai * sa[r + 1][lane];
          const float pr = xr > 0.0f ? 1.0f - __expf(-b2 * xr) : 0.0f;
          const float pd = xd > 0.0f ? 1.0f - __expf(-b2 * xd) : 0.0f;
          br = u0 < pr;
          bd = u1 < pd;
          if (EXACT) {
            const bool amb_r = fabsf(u0 - pr) <= eps;
            const bool amb_d = fabsf(u1 - pd) <= eps;
            if (amb_r || amb_d) {
              const double beta = st->beta, cp = st->cphi, sp = st->sphi;
              const float thi = load_angle(th, static_cast<uint64_t>(i));
              if (amb_r) {
                const uint32_t xn = (static_cast<uint32_t>(lane) + 1u < g.w) ? g.x0 + lane + 1u : g.xh;
                const float thj = load_angle(th, static_cast<uint64_t>(gy) * L + xn);
                const bool e = bond_fp64(thi, thj, rn.w0, beta, cp, sp);
                atomicAdd(&st->n_fp64, 1ull);
                if (e != br) atomicAdd(&st->n_fp32_wrong, 1ull);
                br = e;
              }
              if (amb_d) {
                const uint32_t yn = (r + 1u < g.h) ? gy + 1u : g.yh;
                const float thj = load_angle(th, static_cast<uint64_t>(yn) * L + g.x0 + lane);
                const bool e = bond_fp64(thi, thj, rn.w1, beta, cp, sp);
                atomicAdd(&st->n_fp64, 1ull);
                if (e != bd) atomicAdd(&st->n_fp32_wrong, 1ull);
                bd = e;
              }
            }
          }
          cn = (rn.w2 & 1u) != 0u;
        }
        const uint32_t Rw = __ballot_sync(0xFFFFFFFFu, br);
        const uint32_t Dw = __ballot_sync(0xFFFFFFFFu, bd);
        const uint32_t Cw = __ballot_sync(0xFFFFFFFFu, cn);
        if (lane == 0) {
          sR[r] = Rw;
          sD[r] = Dw;
          d.rplane[static_cast<uint64_t>(tile) * TY + r] = Rw;
          d.dplane[static_cast<uint64_t>(tile) * TY + r] = Dw;
          const uint32_t i0 = gy * L + g.x0;
          if (!d.ragged) {
            d.coin[i0 >> 5] = Cw;
          } else if (Cw) {
            const uint32_t off = i0 & 31u;
            atomicOr(d.coin + (i0 >> 5), Cw << off);
            if (off) atomicOr(d.coin + (i0 >> 5) + 1, Cw >> (32u - off));
          }
        }
      }
    } else {
      for (uint32_t r = threadIdx.x; r < g.h; r += kThreads) {
        sR[r] = d.rplane[static_cast<uint64_t>(tile) * TY + r];
        sD[r] = d.dplane[static_cast<uint64_t>(tile) * TY + r];
      }
    }
    __syncthreads();
    tile_label<TY>(g, L, sR, sD, par, d.label);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// K2: merge across tile edges.  Work item = (tile, j): j < TY is the right
// edge of tile row j, j >= TY the bottom edge of column j - TY.
// ---------------------------------------------------------------------------
// An edge bond is skipped when the previous edge of the same side is active
// and both pairs of endpoints are joined by a direct bond along the edge: the
// previous edge then unites the same two clusters.
template <int TY>
__device__ __forceinline__ bool edge_bond(const LatDesc &d, uint32_t tile,
                                          uint32_t j, uint32_t *a,
                                          uint32_t *b) {
  const uint32_t L = d.L;
  const Tile g = tile_geom<TY>(L, d.ntx, tile);
  const uint64_t base = static_cast<uint64_t>(tile) * TY;
  if (j < static_cast<uint32_t>(TY)) {
    if (j >= g.h) return false;
    const uint32_t bit = g.w - 1u;
    if (!((__ldg(d.rplane + base + j) >> bit) & 1u)) return false;
    if (j > 0 && ((__ldg(d.rplane + base + j - 1) >> bit) & 1u) &&
        ((__ldg(d.dplane + base + j - 1) >> bit) & 1u)) {
      // the neighbouring tile to the right holds column xh at bit 0
      const uint32_t tx = tile % d.ntx;
      const uint32_t tn = tile - tx + (tx + 1u == d.ntx ? 0u : tx + 1u);
      if (__ldg(d.dplane + static_cast<uint64_t>(tn) * TY + j - 1) & 1u) return false;
    }
    const uint32_t y = g.y0 + j;
    *a = y * L + g.x0 + g.w - 1u;
    *b = y * L + g.xh;
    return true;
  }
  const uint32_t c = j - TY;
  if (c >= g.w) return false;
  const uint32_t D = __ldg(d.dplane + base + g.h - 1u);
  if (!((D >> c) & 1u)) return false;
  if (c > 0 && ((D >> (c - 1u)) & 1u) &&
      ((__ldg(d.rplane + base + g.h - 1u) >> (c - 1u)) & 1u)) {
    // the tile below holds row yh as its row 0, same columns
    const uint32_t ty = tile / d.ntx;
    const uint32_t tb = (ty + 1u == d.nty ? 0u : (ty + 1u) * d.ntx) + tile % d.ntx;
    if ((__ldg(d.rplane + static_cast<uint64_t>(tb) * TY) >> (c - 1u)) & 1u) return false;
  }
  *a = (g.y0 + g.h - 1u) * L + g.x0 + c;
  *b = g.yh * L + g.x0 + c;
  return true;
}

template <int TY>
__global__ void __launch_bounds__(kThreads)
    k_merge(const LatDesc *__restrict__ descs,
            const uint32_t *__restrict__ prefix, uint32_t nrep,
            uint32_t nwork) {
  const uint64_t item = static_cast<uint64_t>(blockIdx.x) * kThreads + threadIdx.x;
  const uint64_t per = TY + 32;
  if (item >= static_cast<uint64_t>(nwork) * per) return;
  const uint32_t work = static_cast<uint32_t>(item / per);
  const uint32_t j = static_cast<uint32_t>(item % per);
  const uint32_t rep = find_rep(prefix, nrep, work);
  const LatDesc &d = descs[rep];
  const uint32_t tile = work - __ldg(prefix + rep);
  uint32_t a, b;
  // start from the tile roots: labels of non-root sites are never written
  // here, so after the merge every site still points at its tile root
  if (edge_bond<TY>(d, tile, j, &a, &b))
    gunion(d.label, __ldcg(d.label + a), __ldcg(d.label + b), d.st);
}

// K3: after all unions, every merged tile root re-points at its grandparent
// until its parent is a root.  All merged tile roots jump concurrently, so a
// chain of length d collapses in O(log d) steps per node instead of a walk of
// length d.  Only ancestors are ever written and roots no longer change.
__device__ __forceinline__ void jump(uint32_t *lab, uint32_t x, DevState *st) {
  for (uint32_t it = 0; it < kFindCap; ++it) {
    const uint32_t p = __ldcg(lab + x);
    if (p == x) return;
    const uint32_t gp = __ldcg(lab + p);
    if (gp == p) return;
    __stcg(lab + x, gp);
  }
  atomicOr(&st->err, kErrFindCap);
}

__device__ __forceinline__ void compress(uint32_t *lab, uint32_t a,
                                         DevState *st) {
  // a is an edge site: jump its tile root (its label, unless a is itself a
  // tile root whose entry the merge already moved) and a itself
  const uint32_t t = __ldcg(lab + a);
  jump(lab, t, st);
  jump(lab, a, st);
}

template <int TY>
__global__ void __launch_bounds__(kThreads)
    k_compress(const LatDesc *__restrict__ descs,
               const uint32_t *__restrict__ prefix, uint32_t nrep,
               uint32_t nwork) {
  const uint64_t item = static_cast<uint64_t>(blockIdx.x) * kThreads + threadIdx.x;
  const uint64_t per = TY + 32;
  if (item >= static_cast<uint64_t>(nwork) * per) return;
  const uint32_t work = static_cast<uint32_t>(item / per);
  const uint32_t j = static_cast<uint32_t>(item % per);
  const uint32_t rep = find_rep(prefix, nrep, work);
  const LatDesc &d = descs[rep];
  const uint32_t tile = work - __ldg(prefix + rep);
  uint32_t a, b;
  if (edge_bond<TY>(d, tile, j, &a, &b)) {
    compress(d.label, a, d.st);
    compress(d.label, b, d.st);
  }
}

// ---------------------------------------------------------------------------
// K4: canonical labels, flip, observable sums
// ---------------------------------------------------------------------------
__device__ __forceinline__ int fix22(float v) {
  // v in [-1, 1]: v + 3 lies in [2, 4], whose FP32 grid step is 2^-22, so the
  // bit pattern minus that of 3.0 is round(v * 2^22).
  return __float_as_int(__fadd_rn(v, 3.0f)) - 0x40400000;
}

template <int TY>
constexpr size_t flip_smem() {
  return sizeof(float2) * (TY + 1) * 33;
}

template <int TY, typename AT, bool LABELS_ONLY>
__global__ void __launch_bounds__(kThreads)
    k_flip_measure(const LatDesc *__restrict__ descs,
                   const uint32_t *__restrict__ prefix, uint32_t nrep,
                   uint32_t nwork) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2(*cs)[33] = reinterpret_cast<float2(*)[33]>(smem);
  __shared__ long long red[kWarps][6];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // a thread handles rows r = warp + 8k (k < KR, r <= h): column `lane` of
  // the tile (and of the row below it), and lane 0 also column xh of rows < h
  constexpr int KR = TY / kWarps + 1;

  for (uint32_t work = blockIdx.x; work < nwork; work += gridDim.x) {
    const uint32_t rep = find_rep(prefix, nrep, work);
    const LatDesc &d = descs[rep];
    const uint32_t tile = work - __ldg(prefix + rep);
    const uint32_t L = d.L;
    const Tile g = tile_geom<TY>(L, d.ntx, tile);
    DevState *st = d.st;
    const uint32_t cur = st->cur;
    const float c32 = st->c32;
    const AT *thin = static_cast<const AT *>(d.theta[cur]);
    AT *thout = static_cast<AT *>(d.theta[cur ^ 1u]);
    uint32_t *lab = d.label;
    const bool col_ok = lane < static_cast<int>(g.w);

    // round 1: labels and angles.  Positions of this thread: rows
    // r = warp + 8k (k < KR, r <= h) at column `lane`, and -- for threads
    // t < h -- row t of the column right of the tile (xh).
    uint32_t l0[KR];
    float t0[KR];
    bool v0[KR];
    const bool vh = threadIdx.x < g.h;
    const uint64_t ih = static_cast<uint64_t>(g.y0 + threadIdx.x) * L + g.xh;
    uint32_t lh = 0u;
    float th_h = 0.0f;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const uint32_t r = warp + k * kWarps;
      v0[k] = (r <= g.h) && col_ok;
      const uint64_t row = static_cast<uint64_t>(r < g.h ? g.y0 + r : g.yh) * L;
      l0[k] = 0u;
      t0[k] = 0.0f;
      if (v0[k]) {
        l0[k] = __ldcg(lab + row + g.x0 + lane);
        if (!LABELS_ONLY) t0[k] = load_angle(thin, row + g.x0 + lane);
      }
    }
    if (vh) {
      lh = __ldcg(lab + ih);
      if (!LABELS_ONLY) th_h = load_angle(thin, ih);
    }
    // round 2: one more hop (the tile root's entry)
    uint32_t p0[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) p0[k] = v0[k] ? __ldcg(lab + l0[k]) : 0u;
    const uint32_t ph = vh ? __ldcg(lab + lh) : 0u;
    // round 3: where the tile root was merged, confirm the next node is the
    // root (the usual case after k_compress) or finish the find
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      if (v0[k] && p0[k] != l0[k]) {
        const uint32_t q = __ldcg(lab + p0[k]);
        l0[k] = (q == p0[k]) ? q : gfind_ro(lab, q, st);
      }
    }
    if (vh && ph != lh) {
      const uint32_t q = __ldcg(lab + ph);
      lh = (q == ph) ? q : gfind_ro(lab, q, st);
    }
    // l0 / lh now hold the roots; own sites get their canonical label
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const uint32_t r = warp + k * kWarps;
      if (v0[k] && r < g.h)
        __stcg(lab + static_cast<uint64_t>(g.y0 + r) * L + g.x0 + lane, l0[k]);
    }
    if (LABELS_ONLY) continue;
    // round 4: coins of the roots
    uint32_t f0[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k)
      f0[k] = v0[k] ? (__ldg(d.coin + (l0[k] >> 5)) >> (l0[k] & 31u)) & 1u : 0u;
    const uint32_t fh = vh ? (__ldg(d.coin + (lh >> 5)) >> (lh & 31u)) & 1u : 0u;
    // flip, store, and cos/sin of the new angles into shared memory
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const uint32_t r = warp + k * kWarps;
      if (v0[k]) {
        float nv = t0[k];
        if (f0[k]) {
          const AT sv = store_value<AT>(wrap_angle(__fadd_rn(c32, -t0[k])));
          nv = stored_float<AT>(sv);
          if (r < g.h) thout[static_cast<uint64_t>(g.y0 + r) * L + g.x0 + lane] = sv;
        } else if (r < g.h) {
          thout[static_cast<uint64_t>(g.y0 + r) * L + g.x0 + lane] = store_value<AT>(t0[k]);
        }
        float s, co;
        sincosf(nv, &s, &co);
        cs[r][lane] = make_float2(co, s);
      }
    }
    if (vh) {
      float nv = th_h;
      if (fh) nv = stored_float<AT>(store_value<AT>(wrap_angle(__fadd_rn(c32, -th_h))));
      float s, co;
      sincosf(nv, &s, &co);
      cs[threadIdx.x][g.w] = make_float2(co, s);
    }
    __syncthreads();
    // terms of the tile's own sites
    int acc[6] = {0, 0, 0, 0, 0, 0};
    if (col_ok) {
      for (uint32_t r = warp; r < g.h; r += kWarps) {
        const float2 a = cs[r][lane], rr = cs[r][lane + 1], dd = cs[r + 1][lane];
        acc[0] += fix22(a.x);
        acc[1] += fix22(a.y);
        acc[2] += fix22(fmaf(a.x, rr.x, a.y * rr.y));
        acc[3] += fix22(fmaf(a.y, rr.x, -(a.x * rr.y)));
        acc[4] += fix22(fmaf(a.x, dd.x, a.y * dd.y));
        acc[5] += fix22(fmaf(a.y, dd.x, -(a.x * dd.y)));
      }
    }
    long long v[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      v[k] = acc[k];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1)
        v[k] += __shfl_down_sync(0xFFFFFFFFu, v[k], off);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 6; ++k) red[warp][k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < 6) {
      long long sum = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) sum += red[w][threadIdx.x];
      atomicAdd(reinterpret_cast<unsigned long long *>(
                    d.acc + (tile % kSlots) * kAccStride + threadIdx.x),
                static_cast<unsigned long long>(sum));
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// axis of sweep t and the FP32 constants derived from it and beta
// ---------------------------------------------------------------------------
__device__ inline void set_sweep_params(DevState *st, uint32_t t, double beta,
                                        uint32_t k0, uint32_t k1) {
  const Words4 w = philox4x32_10(0u, 0u, t, kDomAxis, k0, k1);
  const uint64_t bits = (static_cast<uint64_t>(w.w0) << 32) | w.w1;
  const double u = static_cast<double>(bits >> 11) * 0x1p-53;
  const double phi = __dmul_rn(6.283185307179586, u);
  double s, c;
  sincos(phi, &s, &c);
  const double C = fmod(__dadd_rn(3.141592653589793, __dmul_rn(2.0, phi)),
                        6.283185307179586);
  float c32 = __double2float_rn(C);
  if (c32 >= two_pi_f()) c32 = 0.0f;
  st->t = t;
  st->beta = beta;
  st->cphi = c;
  st->sphi = s;
  st->cphi32 = __double2float_rn(c);
  st->sphi32 = __double2float_rn(s);
  st->c32 = c32;
  st->beta2_32 = __double2float_rn(2.0 * beta);
  // band half-width: 4x the error bound of the FP32 evaluation of u - p
  st->eps = __double2float_rn(4.0 * (2.0 * beta * 2.0e-6 + 3.0e-7) + 0x1p-24);
}

// K5: one warp per lattice
static __global__ void k_finalize(const LatDesc *__restrict__ descs, uint32_t nrep) {
  const uint32_t rep = blockIdx.x;
  if (rep >= nrep) return;
  const LatDesc &d = descs[rep];
  DevState *st = d.st;
  const int lane = threadIdx.x;
  long long v[6] = {0, 0, 0, 0, 0, 0};
  for (int s = lane; s < kSlots; s += 32) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      v[k] += d.acc[s * kAccStride + k];
      d.acc[s * kAccStride + k] = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
      v[k] += __shfl_down_sync(0xFFFFFFFFu, v[k], off);
  }
  if (lane != 0) return;
  const double n = static_cast<double>(d.L) * static_cast<double>(d.L);
  double S[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) S[k] = static_cast<double>(v[k]) / kFixScale;
  const double beta = st->beta;
  ObsRecord o;
  o.mx = S[0] / n;
  o.my = S[1] / n;
  o.m2 = o.mx * o.mx + o.my * o.my;
  o.ex = S[2] / n;
  o.sx = S[3] / n;
  o.ey = S[4] / n;
  o.sy = S[5] / n;
  o.energy_per_site = -(S[2] + S[4]) / n;
  o.upsilon = o.ex - beta * n * o.sx * o.sx;  // Eq. (4), J = 1, T = 1/beta
  o.beta = beta;
  o.sweep = st->t;
  d.rec[st->rec_count % d.rec_cap] = o;
  st->rec_count += 1;
  double nb = beta;
  if (st->pcc_on) {
    st->pcc_acc += beta * o.upsilon;
    st->pcc_count += 1;
    if (st->pcc_count >= st->pcc_block) {
      const double mean = st->pcc_acc / static_cast<double>(st->pcc_block);
      double db = st->pcc_dbeta0;
      if (st->pcc_halve) db = ldexp(db, -static_cast<int>(st->pcc_k / st->pcc_halve));
      nb = (mean < st->pcc_target) ? beta + db : beta - db;
      st->pcc_acc = 0.0;
      st->pcc_count = 0;
    }
    st->pcc_k += 1;
  }
  st->cur ^= 1u;
  set_sweep_params(st, st->t + 1u, nb, d.key0, d.key1);
}

// ---------------------------------------------------------------------------
// initialisation and host-driven state updates
// ---------------------------------------------------------------------------
template <typename AT>
__global__ void k_init_angles(LatDesc d, int ordered) {
  const uint64_t n = static_cast<uint64_t>(d.L) * d.L;
  AT *th = static_cast<AT *>(d.theta[0]);
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
       i < n; i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    float v = 0.0f;
    if (!ordered) {
      const Words4 w = philox4x32_10(static_cast<uint32_t>(i),
                                     static_cast<uint32_t>(i >> 32),
                                     0xFFFFFFFFu, kDomInit, d.key0, d.key1);
      const float step = 6.2831854820251465f * 0x1p-24f;
      v = __fmul_rn(static_cast<float>(w.w0 >> 8), step);
      if (v >= two_pi_f()) v = 0.0f;
    }
    th[i] = store_value<AT>(v);
  }
}

static __global__ void k_init_state(LatDesc d, double beta) {
  DevState *st = d.st;
  st->cur = 0;
  st->pcc_on = 0;
  st->pcc_block = 1;
  st->pcc_halve = 0;
  st->pcc_count = 0;
  st->pcc_target = 0.0;
  st->pcc_dbeta0 = 0.0;
  st->pcc_acc = 0.0;
  st->pcc_k = 0;
  st->rec_count = 0;
  st->n_fp64 = 0;
  st->n_fp32_wrong = 0;
  st->err = 0;
  set_sweep_params(st, 0u, beta, d.key0, d.key1);
}

static __global__ void k_set_pcc(DevState *st, uint32_t on, double target,
                          double dbeta0, uint32_t halve, uint32_t block) {
  st->pcc_on = on;
  if (on) {
    st->pcc_target = target;
    st->pcc_dbeta0 = dbeta0;
    st->pcc_halve = halve;
    st->pcc_block = block;
  }
}

}  // namespace xyk
