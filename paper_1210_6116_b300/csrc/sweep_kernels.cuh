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
//                  step (Sec. 2) and the random axis of the next sweep.  At
//                  fixed beta a single lattice runs this work in block 0 of
//                  the next sweep's k_bond_label instead (kCtlDraw), and
//                  k_finalize only closes each API call with the last record.
//
// Layouts (per lattice, N = L*L, i = y*L + x):
//   theta[2]  angle double buffer (FP32, FP16 or u16); the sweep reads theta[cur]
//             and writes theta[cur ^ 1], so halo reads never race with flips.
//   label     N uint32.
//   rplane,   tile-major bond bit planes: word (tile*TY + r) holds the right
//   dplane    (down) bonds of tile row r, bit c = column x0 + c.
//   coin      linear bit array, bit i = coin of site i (read only for roots).
//   acc       kSlots x kAccStride int64 accumulators of the fixed-point sums.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

#include <type_traits>

#include "philox.cuh"

namespace xyk {

constexpr int kThreads = 256;          // 8 warps per tile CTA
constexpr int kWarps = kThreads / 32;
constexpr int kSlots = 64;             // accumulator slots per lattice
constexpr int kAccStride = 16;         // int64 per slot (6, or 14 with xi; [15] flips)
constexpr int kFlipSlot = 15;          // slot entry counting the reflected sites
// default bound on the iterations of any global find / union / jump loop
// (LatDesc::find_cap; a test may lower it to make the bound run out)
constexpr uint32_t kFindCap = 1u << 22;

// error bits recorded in DevState::err
constexpr uint32_t kErrFindCap = 1u;
constexpr uint32_t kErrUnionCap = 2u;
constexpr uint32_t kErrLinkCap = 4u;  // more links than the tile's link slots
constexpr uint32_t kErrBounds = 8u;   // bounds-checked build: a global index out of range

// The bounds-checked build (compiled with -DXY_BOUNDS_CHECK) tests every
// global index that comes from data (a label value used as an address, a
// link read back): one at or past the array's size records kErrBounds and
// is replaced by 0, so the access stays inside the array, the launch
// completes and the next synchronising call returns XY_EINTERNAL.  In the
// normal build chk() is the identity: those indices are in range by
// construction (every label is a site index of its own lattice).
#ifdef XY_BOUNDS_CHECK
constexpr bool kBoundsCheck = true;
#else
constexpr bool kBoundsCheck = false;
#endif

// Fixed-point scale of the observable sums: each FP32 term in [-1, 1] is
// rounded to a multiple of 2^-22 and summed exactly in integers.
constexpr double kFixScale = 4194304.0;  // 2^22

struct ObsRecord {  // identical layout to xy_obs
  double energy_per_site, m2, mx, my, ex, sx, ey, sy, upsilon, beta;
  uint64_t sweep;
  double chik;
  uint64_t flipped;
};

// Parameters of one sweep: its index, the angle buffer it reads, beta and
// the random axis r of Sec. 2 with the values derived from it.
struct SweepParams {
  uint32_t t;      // sweep counter
  uint32_t cur;    // theta buffer holding the angles the sweep reads
  double beta;
  double cphi, sphi;     // axis of sweep t (FP64)
  float cphi32, sphi32;  // FP32 copies
  float c32;             // reflection constant: theta' = c32 - theta (mod 2pi)
  float beta2_32;        // 2 beta in FP32
  float eps;             // half-width of the FP32 error band of exact mode
  uint32_t seed_site;    // Wolff update t: the site whose cluster is reflected
};

// Bits of K1's `ctl` argument (single-lattice launches; 0 elsewhere).  The
// parameters of a sweep are in p[par]; with kCtlDraw the launch has one
// block more than tiles, and its block 0 writes the parameters of the next
// sweep into p[par ^ 1] (no kernel of this sweep reads that slot), after,
// with kCtlRecord, appending the record of the previous sweep, whose
// parameters that slot still holds.  This folds k_finalize into the next
// sweep's K1 for runs at fixed beta.
constexpr uint32_t kCtlPar = 1u, kCtlDraw = 2u, kCtlRecord = 4u;
// k_finalize's `mode`: 0 the full step (record, PCC, next parameters into
// both slots); kFinRecord | par: the record of the sweep in p[par], then
// p[par] = p[par ^ 1], so that both slots again hold the next sweep's.
constexpr uint32_t kFinRecord = 2u;

struct DevState {
  // p[0] == p[1] between API calls; within a fixed-beta call the slots
  // alternate by sweep parity (see kCtlDraw)
  SweepParams p[2];
  uint32_t pcc_on;
  // helicity-modulus PCC
  uint32_t pcc_block, pcc_halve, pcc_count;
  uint32_t quant;  // 1: u16 angles, axis on the reflection grid
  double pcc_target, pcc_dbeta0, pcc_acc;
  uint64_t pcc_k;
  // records
  uint64_t rec_count;
  // diagnostics
  unsigned long long n_fp64, n_fp32_wrong;
  uint32_t err;
};

struct LatDesc {
  uint32_t L, ntx, nty, ntiles;
  uint32_t key0, key1, rec_cap, ragged;
  uint64_t Lmagic;     // ceil(2^64 / L): x / L == umul64hi(x, Lmagic) for x < 2^32
  uint64_t ntx_magic;  // ceil(2^64 / ntx) (0 for ntx = 1): the same exact division by ntx
  double inv_n;     // 1 / L^2
  uint32_t xi;     // 1: accumulate the Fourier sums of chik
  uint32_t wolff;  // 1: Wolff single-cluster update (reflect the seed's cluster)
  uint32_t find_cap;  // iteration bound of the global find / union / jump loops
  uint32_t link_cap;  // link slots a tile may fill per sweep (at most TY + 32)
  const float2 *wave;  // [L]: (cos, sin)(2 pi x / L), used when xi
  void *theta[2];
  uint32_t *label;
  uint32_t *rplane, *dplane;
  uint32_t *edge;  // per tile: labels of its left/right columns, top/bottom rows
  uint32_t *links;       // per tile, TY + 32 slots: tile roots its edge items linked
  uint32_t *link_count;  // per tile: the slots used this sweep (reset by K1)
  uint32_t *coin;
  long long *acc;
  DevState *st;
  ObsRecord *rec;
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t chk(uint32_t i, uint64_t n, DevState *st) {
  if constexpr (kBoundsCheck) {
    if (i >= n) {
      atomicOr(&st->err, kErrBounds);
      return 0u;
    }
  }
  return i;
}

__device__ __forceinline__ float two_pi_f() { return 6.2831854820251465f; }
__device__ __forceinline__ float pi_f() { return 3.14159274101257324f; }

template <typename AT>
__device__ __forceinline__ float load_angle(const AT *p, uint64_t i);
// Angles are read once per kernel and the sweep's working set exceeds L2, so
// they load evict-first and leave L2 to the labels, planes and edge tables
// the next kernels gather from (L = 4096: -1 us per sweep).
template <>
__device__ __forceinline__ float load_angle<float>(const float *p, uint64_t i) {
  return __ldcs(p + i);
}
template <>
__device__ __forceinline__ float load_angle<__half>(const __half *p,
                                                    uint64_t i) {
  return __half2float(__ldcs(p + i));
}
// u16 fixed point: the stored q itself (exact in FP32); the angle is
// q 2pi / 65536, see angle_f32 / angle_f64 below
template <>
__device__ __forceinline__ float load_angle<uint16_t>(const uint16_t *p,
                                                      uint64_t i) {
  return static_cast<float>(__ldcs(p + i));
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
template <>
__device__ __forceinline__ uint16_t store_value<uint16_t>(float v) {
  return static_cast<uint16_t>(static_cast<uint32_t>(v));  // v is an exact q
}
// the storage word of a raw value that is already in the storage format and
// in range (a loaded angle, or a reflected one from reflect below): no
// rounding or wrap left to do
template <typename AT>
__device__ __forceinline__ AT store_exact(float raw) {
  return store_value<AT>(raw);
}
template <>
__device__ __forceinline__ __half store_exact<__half>(float raw) {
  return __float2half_rn(raw);  // exact: raw is a half value
}

// Kernels hold every stored angle as a float that equals the stored value
// exactly ("raw": the FP32 angle, the FP16 angle widened, or u16's q).  The
// traits below turn a raw value into radians and apply the reflection.
template <typename AT>
__device__ __forceinline__ float angle_f32(float raw) {  // radians, FP32
  return raw;
}
template <>
__device__ __forceinline__ float angle_f32<uint16_t>(float raw) {
  return __fmul_rn(raw, 6.2831854820251465f * 0x1p-16f);  // q 2pi_f 2^-16
}
template <typename AT>
__device__ __forceinline__ double angle_f64(float raw) {  // radians, FP64
  return static_cast<double>(raw);
}
template <>
__device__ __forceinline__ double angle_f64<uint16_t>(float raw) {
  return __dmul_rn(static_cast<double>(raw), 6.283185307179586 * 0x1p-16);
}
// reflected raw value: wrap(c - theta) in FP32, rounded to the storage format;
// u16: (Cq - q) mod 65536 in integers (c holds Cq)
template <typename AT>
__device__ __forceinline__ float reflect(float raw, float c);
template <>
__device__ __forceinline__ float reflect<float>(float raw, float c) {
  return wrap_angle(__fadd_rn(c, -raw));
}
template <>
__device__ __forceinline__ float reflect<__half>(float raw, float c) {
  return __half2float(store_value<__half>(wrap_angle(__fadd_rn(c, -raw))));
}
template <>
__device__ __forceinline__ float reflect<uint16_t>(float raw, float c) {
  const uint32_t q = static_cast<uint32_t>(raw), cq = static_cast<uint32_t>(c);
  return static_cast<float>((cq + 65536u - q) & 0xFFFFu);
}
// sin and cos of an angle x with |x| <= 8 (stored angles lie in [0, 2 pi)),
// for the observables.  Cody-Waite reduction by pi/2 (W. J. Cody and
// W. Waite, Software Manual for the Elementary Functions, 1980): q is the
// integer nearest x 2/pi, r = x - q P1 - q P2 with P1 the float nearest pi/2
// and P2 the float nearest pi/2 - P1.  The first FMA is exact (q <= 5: the
// difference is a multiple of 2^-24 below 1 in magnitude), the second rounds
// once (<= 3e-8), and pi/2 - P1 - P2 = -1.8e-15 is negligible.  Then
// minimax polynomials on |r| <= pi/4, fitted for this routine by the Remez
// exchange algorithm (weighted absolute error, coefficients rounded to
// FP32): sin r = r + r^3 (S0 + S1 r^2 + S2 r^4) with truncation error
// <= 1.8e-9, cos r = 1 + r^2 (C0 + C1 r^2 + C2 r^4 + C3 r^6) with <= 5.4e-11;
// Horner with FMAs, and the quadrant q mod 4 by swapping and sign flips.
// Absolute error <= 1e-7 for both (the tests measure it against FP64); the
// SFU's __sincosf (~3.6e-7) is not accurate enough for the observable
// tolerances.
// The polynomials at the reduced argument r (|r| <= pi/4), moved to quadrant
// iq mod 4: (sin, cos)(r + iq pi/2).
__device__ __forceinline__ void sincos_quadrant(float r, uint32_t iq, float *s, float *c) {
  const float r2 = r * r;
  float ps = fmaf(r2, -0x1.98da66p-13f, 0x1.1105b4p-7f);  // S2 r^2 + S1
  ps = fmaf(ps, r2, -0x1.55554p-3f);                      // .. + S0
  const float sr = fmaf(ps * r2, r, r);
  float pc = fmaf(r2, 0x1.99343p-16f, -0x1.6c087ep-10f);  // C3 r^2 + C2
  pc = fmaf(pc, r2, 0x1.55553ep-5f);                      // .. + C1
  pc = fmaf(pc, r2, -0.5f);                               // .. + C0
  const float cr = fmaf(pc, r2, 1.0f);
  // (sin, cos)(r + q pi/2) = (sr, cr), (cr, -sr), (-sr, -cr), (-cr, sr)
  const bool odd = (iq & 1u) != 0u;
  *s = __uint_as_float(__float_as_uint(odd ? cr : sr) ^ ((iq & 2u) << 30));
  *c = __uint_as_float(__float_as_uint(odd ? sr : cr) ^ (((iq + 1u) & 2u) << 30));
}
__device__ __forceinline__ void sincos_cw(float x, float *s, float *c) {
  constexpr float kTwoOverPi = 0x1.45f306p-1f;  // float nearest 2/pi
  constexpr float kP1 = 0x1.921fb6p+0f;         // float nearest pi/2
  constexpr float kP2 = -0x1.777a5cp-25f;       // float nearest pi/2 - kP1
  constexpr float kRound = 0x1.8p23f;           // 1.5 2^23: adds round to integers
  const float t = fmaf(x, kTwoOverPi, kRound);   // kRound + q
  const float q = t - kRound;                    // exact
  float r = fmaf(-q, kP1, x);
  r = fmaf(-q, kP2, r);
  sincos_quadrant(r, __float_as_uint(t), s, c);  // the low bits of t: q mod 4
}
template <typename AT>
__device__ __forceinline__ void sin_cos(float raw, float *s, float *c) {
  sincos_cw(raw, s, c);
}
template <>
__device__ __forceinline__ void sin_cos<uint16_t>(float raw, float *s, float *c) {
  // angle q 2pi / 65536 = n pi/2 + m pi/32768 with n the nearest integer to
  // q / 16384 and |m| <= 8192, both exact integers; r = m pi/32768 by one
  // FMA over pi/32768 split in two floats (sincos_cw's P1, P2 times 2^-14):
  // within ~3e-8 of the exact remainder, and over all 65536 q the result is
  // within 6.5e-8 of FP64 cos and sin
  const int q = static_cast<int>(raw);
  const int n = (q + 8192) >> 14;
  const float m = static_cast<float>(q - (n << 14));
  const float r = fmaf(m, 0x1.921fb6p-14f, m * -0x1.777a5cp-39f);
  sincos_quadrant(r, static_cast<uint32_t>(n), s, c);
}

// projection s.r in FP32 from the stored angle; sin/cos through the SFU on
// the centred argument theta - pi_f in [-pi, pi)
__device__ __forceinline__ float project32(float th, float cphi, float sphi) {
  float s, c;
  __sincosf(__fadd_rn(th, -pi_f()), &s, &c);  // s = -sin th, c = -cos th
  return -fmaf(c, cphi, s * sphi);
}

// FP64 projection exactly as the rule defines it: cos(th) cphi + sin(th) sphi
__device__ __forceinline__ double project64(double th, double cphi,
                                            double sphi) {
  double s, c;
  sincos(th, &s, &c);
  return __dadd_rn(__dmul_rn(c, cphi), __dmul_rn(s, sphi));
}

// Programmatic dependent launch: let the next kernel on the stream be
// scheduled once every block of this grid runs, and wait for the previous
// kernel's grid (and its memory) before touching anything it writes.  Both
// are no-ops for a kernel launched without the attribute.  Every sweep
// kernel calls this (or pdl_prologue_last) before its first read of mutable
// data.
__device__ __forceinline__ void pdl_prologue() {
  cudaTriggerProgrammaticLaunchCompletion();
  cudaGridDependencySynchronize();
}

// The same with the trigger after the wait, for the first and last kernels
// of a sweep (K1 and K4): the merge is launched only once the previous K4
// has completed, and the next sweep's K1 only once this sweep's compress has.
// With every kernel triggering first, launched grids that wait for their
// predecessors pile up ever further ahead of the running one, and small
// lattices ran slower (L = 512: 26.5 us per sweep, against 23.3 with K4's
// trigger late and 22.4 with both; L >= 1024 unchanged).
__device__ __forceinline__ void pdl_prologue_last() {
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
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

// FULL: every tile of the lattice is a whole 32 x TY (L a multiple of 32 and
// of TY), so width and height are compile-time constants and the ragged-edge
// tests of the kernels fold away.
template <int TY, bool FULL = false>
__device__ __forceinline__ Tile tile_geom(uint32_t L, uint32_t ntx, uint64_t ntx_magic,
                                          uint32_t tile) {
  Tile g;
  // tile / ntx as a multiply-high by ceil(2^64 / ntx): exact for 32-bit
  // operands (the error term stays below 2^-32 < 1 / ntx); ceil(2^64 / 1)
  // does not fit, so one tile column is its own case (ntx_magic = 0)
  const uint32_t ty = ntx == 1u ? tile : static_cast<uint32_t>(__umul64hi(tile, ntx_magic));
  const uint32_t tx = tile - ty * ntx;
  g.x0 = tx * 32u;
  g.y0 = ty * static_cast<uint32_t>(TY);
  g.w = FULL ? 32u : min(32u, L - g.x0);
  g.h = FULL ? static_cast<uint32_t>(TY) : min(static_cast<uint32_t>(TY), L - g.y0);
  g.xh = (g.x0 + g.w == L) ? 0u : g.x0 + g.w;  // column right of the tile
  g.yh = (g.y0 + g.h == L) ? 0u : g.y0 + g.h;  // row below the tile
  return g;
}

// ---------------------------------------------------------------------------
// bond decision
// ---------------------------------------------------------------------------
// FP64 rule, operation for operation: x = a_i a_j; active iff x > 0 and
// ((w >> 1) + 1/2) 2^-31 < 1 - exp(-2 beta x).
static __device__ __noinline__ bool bond_fp64(double th_i, double th_j, uint32_t word,
                                              double beta, double cphi, double sphi) {
  const double ai = project64(th_i, cphi, sphi);
  const double aj = project64(th_j, cphi, sphi);
  const double x = __dmul_rn(ai, aj);
  if (!(x > 0.0)) return false;
  const double p = __dsub_rn(1.0, exp(__dmul_rn(__dmul_rn(-2.0, beta), x)));
  const double u = __dmul_rn(__dadd_rn(static_cast<double>(word >> 1), 0.5),
                             0x1p-31);
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

// Final find after the scan and the unions: almost every site is at most one
// hop from its root, so two loads settle it and only a longer chain loops
// (K1 at L = 4096: 123.6 -> 119.4 us against the looping find).
__device__ __forceinline__ uint32_t sfind2(volatile uint32_t *par, uint32_t a) {
  const uint32_t p = par[a];
  const uint32_t pp = par[p];
  if (pp != p) return sfind(par, pp);
  return p;
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
__device__ __forceinline__ uint32_t gfind_halve(uint32_t *lab, uint64_t n, uint32_t a,
                                                DevState *st, uint32_t cap) {
  for (uint32_t it = 0; it < cap; ++it) {
    const uint32_t p = chk(__ldcg(lab + chk(a, n, st)), n, st);
    if (p == a) return a;
    const uint32_t gp = chk(__ldcg(lab + p), n, st);
    if (gp != p) __stcg(lab + a, gp);  // gp is an ancestor: safe to skip p
    a = gp;
  }
  atomicOr(&st->err, kErrFindCap);
  return a;
}

// A successful link of root a is appended to the calling tile's link slots
// (at most one per call, so the tile's edge-item count bounds them; one
// counter per tile keeps the appends from piling onto one address):
// k_compress jumps exactly those roots.
__device__ __forceinline__ void gunion(uint32_t *lab, uint64_t n, uint32_t a, uint32_t b,
                                       DevState *st, uint32_t fcap, uint32_t *links,
                                       uint32_t *count, uint32_t cap) {
  a = gfind_halve(lab, n, a, st, fcap);
  b = gfind_halve(lab, n, b, st, fcap);
  for (uint32_t it = 0; a != b; ++it) {
    if (it >= fcap) {
      atomicOr(&st->err, kErrUnionCap);
      return;
    }
    if (a < b) {
      const uint32_t tmp = a;
      a = b;
      b = tmp;
    }
    const uint32_t old = atomicCAS(lab + chk(a, n, st), a, b);
    if (old == a) {
      const uint32_t k = atomicAdd(count, 1u);
      if (k < cap) links[k] = a;
      else atomicOr(&st->err, kErrLinkCap);
      return;
    }
    a = gfind_halve(lab, n, old, st, fcap);
    b = gfind_halve(lab, n, b, st, fcap);
  }
}

// ---------------------------------------------------------------------------
// K1 layout: a CTA owns one 32 x TY tile; warp w owns the band of B = TY/8
// consecutive rows starting at r0 = w*B, lane = column.  Projections stay in
// registers (the right neighbour by shuffle, the row below from the next
// iteration).  Labels come from a row scan inside the band: each row run
// takes the smallest root among the runs above it that it touches (a
// segmented minimum over the run's lanes), and only a run that touches two
// different upper components causes a union.  Bands are then joined across
// their boundary rows, and every site gets the root of its run.
//
// Union-find nodes are tile-local indices r*32 + c of run starts; par[] lives
// in shared memory and every link points to a smaller index, so the root of a
// component is its smallest site, which is also its smallest global index.
// ---------------------------------------------------------------------------
constexpr uint32_t kNoRoot = 0xFFFFFFFFu;

// Edge table of a 32 x TY tile, written by K1 and read by the merge: the
// tile-local root (a global site index) of every site on its boundary, as
// [left column: TY][right column: TY][top row: 32][bottom row: 32].  The
// merge reads these compactly instead of one sector per label of a column.
template <int TY>
__host__ __device__ constexpr uint32_t edge_words() {
  return 2u * TY + 64u;
}

// lanes of the run containing `lane`: [start, end]
__device__ __forceinline__ uint32_t run_start_of(uint32_t starts, int lane) {
  return 31u - __clz(starts & (0xFFFFFFFFu >> (31 - lane)));
}

// One row of the band scan.  up = the scan root above this lane if the
// vertical bond from the previous row is active, else kNoRoot.  The run's
// root is the smallest `up` over its lanes (or its own start node when no
// lane is connected above), found by a segmented suffix minimum.  Every other
// upper root that the run touches is an equivalence, appended to the warp's
// pair list (warp-aggregated, no atomics) and united later by all threads at
// once; only a full list falls back to an immediate union.  Returns the
// lane's scan root.
template <int CAP>
__device__ __forceinline__ uint32_t scan_row(uint32_t *par, uint32_t *pairs,
                                             uint32_t &npairs, uint32_t *runmin,
                                             uint32_t r, uint32_t starts,
                                             uint32_t up, int lane) {
  const uint32_t s = run_start_of(starts, lane);
  // minimum of `up` over the run, gathered in the run start's slot of the
  // warp's scratch (every slot holds kNoRoot between rows)
  if (up != kNoRoot) atomicMin(runmin + s, up);
  __syncwarp();
  // m_run <= up on every lane of the run, so need implies m_run != kNoRoot
  const uint32_t m_run = runmin[s];
  __syncwarp();
  if (static_cast<uint32_t>(lane) == s) runmin[s] = kNoRoot;
  const uint32_t node = r * 32u + s;
  const uint32_t root = (m_run == kNoRoot) ? node : m_run;
  const uint32_t prev_up = __shfl_up_sync(0xFFFFFFFFu, up, 1);
  const bool need = up != kNoRoot && up != m_run &&
                    !(static_cast<uint32_t>(lane) > s && prev_up == up);
  const uint32_t mask = __ballot_sync(0xFFFFFFFFu, need);
  if (mask) {
    const uint32_t off = npairs + __popc(mask & ((1u << lane) - 1u));
    if (need) {
      if (off < static_cast<uint32_t>(CAP)) pairs[off] = (up << 16) | m_run;
      else sunion(par, up, m_run);
    }
    npairs += __popc(mask);
  }
  if (static_cast<uint32_t>(lane) == s) par[node] = root;
  __syncwarp();  // the run node is read by other lanes from the next row on
  return root;
}

// capacity of a warp's equivalence-pair list
template <int TY>
__host__ __device__ constexpr int pair_cap() {
  return 16 * (TY / kWarps);
}

template <int TY>
constexpr size_t bond_label_smem() {
  return sizeof(uint32_t) * (TY * 32 + 2 * TY + kWarps * pair_cap<TY>() + kWarps * 32);
}

// ---------------------------------------------------------------------------
// axis of sweep t and the FP32 constants derived from it and beta
// ---------------------------------------------------------------------------
// The part of sweep t's parameters that does not depend on beta: the axis,
// the reflection constant and the Wolff seed site.
struct Axis {
  double c, s;         // cos, sin of the axis angle (FP64)
  float c32;           // reflection constant (u16: Cq)
  uint32_t seed_site;  // Wolff: the site whose cluster is reflected
};

__device__ inline Axis draw_axis(uint32_t quant, uint32_t t, uint32_t k0, uint32_t k1,
                                 uint32_t L) {
  const Words4 w = philox4x32_10(0u, 0u, t, kDomAxis, k0, k1);
  Axis a;
  // seed site of a Wolff update: word 2 scaled to 0 .. N-1 (N = L^2 <= 2^32)
  a.seed_site = static_cast<uint32_t>(
      (static_cast<uint64_t>(w.w2) * (static_cast<uint64_t>(L) * L)) >> 32);
  const uint64_t bits = (static_cast<uint64_t>(w.w0) << 32) | w.w1;
  if (quant) {
    // u16 angles: the axis on the reflection grid, phi_q = pi m / 65536 with
    // m = phi mod pi floored to the grid, and Cq = m + 32768 (mod 65536), so
    // that pi + 2 phi_q = Cq 2pi / 65536 and the flip is q -> Cq - q
    const uint32_t m = static_cast<uint32_t>(bits >> 47) & 0xFFFFu;
    sincospi(static_cast<double>(m) * 0x1p-16, &a.s, &a.c);
    a.c32 = static_cast<float>((m + 32768u) & 0xFFFFu);
  } else {
    const double u = static_cast<double>(bits >> 11) * 0x1p-53;
    const double phi = __dmul_rn(6.283185307179586, u);
    sincos(phi, &a.s, &a.c);
    // C = (pi + 2 phi) mod 2pi.  pi + 2 phi lies in [pi, 5pi) and both
    // subtractions are exact (Sterbenz), so this is fmod's result exactly.
    const double two_pi = 6.283185307179586;
    double C = __dadd_rn(3.141592653589793, __dmul_rn(2.0, phi));
    if (C >= 2.0 * two_pi) C = __dsub_rn(C, 2.0 * two_pi);
    else if (C >= two_pi) C = __dsub_rn(C, two_pi);
    a.c32 = __double2float_rn(C);
    if (a.c32 >= two_pi_f()) a.c32 = 0.0f;
  }
  return a;
}

__device__ inline void set_sweep_params(SweepParams *p, uint32_t quant, uint32_t t,
                                        uint32_t cur, double beta, const Axis &a) {
  p->t = t;
  p->cur = cur;
  p->beta = beta;
  p->cphi = a.c;
  p->sphi = a.s;
  p->cphi32 = __double2float_rn(a.c);
  p->sphi32 = __double2float_rn(a.s);
  p->c32 = a.c32;
  p->seed_site = a.seed_site;
  p->beta2_32 = __double2float_rn(2.0 * beta);
  // band half-width: 4x the error bound of the FP32 evaluation of u - p;
  // u16 adds <= 4.2e-7 per projection for the FP32 angle q 2pi_f 2^-16
  const double dx = quant ? 3.0e-6 : 2.0e-6;
  p->eps = __double2float_rn(4.0 * (2.0 * beta * dx + 3.0e-7) + 0x1p-24);
}

// ---------------------------------------------------------------------------
// the per-sweep record (Eqs. (3)-(6), FP64)
// ---------------------------------------------------------------------------
// Called by one whole warp whose lane k holds S_k, the fixed-point sum of
// accumulator entry k % 16 over all slots.  Lane 0 appends the record of
// sweep t to the ring and returns it (the other lanes' return is unused).
// k_finalize and the folded record in K1 both call this, so the two give
// bit-identical records.
__device__ __forceinline__ ObsRecord append_record(const LatDesc &d, DevState *st,
                                                   long long tot, double beta, uint32_t t,
                                                   uint64_t rec_count) {
  const int lane = threadIdx.x & 31;
  const double x = static_cast<double>(tot) * (1.0 / kFixScale);  // S_k
  const double y = x * d.inv_n;                                     // S_k / N
  double sq = (lane >= 6 && lane < 14) ? x * x : 0.0;  // |F|^2 terms of chik
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xFFFFFFFFu, sq, off);
  const double mx = __shfl_sync(0xFFFFFFFFu, y, 0), my = __shfl_sync(0xFFFFFFFFu, y, 1);
  const double ex = __shfl_sync(0xFFFFFFFFu, y, 2), sx = __shfl_sync(0xFFFFFFFFu, y, 3);
  const double ey = __shfl_sync(0xFFFFFFFFu, y, 4), sy = __shfl_sync(0xFFFFFFFFu, y, 5);
  const double x2 = __shfl_sync(0xFFFFFFFFu, x, 2), x4 = __shfl_sync(0xFFFFFFFFu, x, 4);
  const long long nf = __shfl_sync(0xFFFFFFFFu, tot, kFlipSlot);
  ObsRecord o{};
  if (lane == 0) {
    const double n = static_cast<double>(d.L) * static_cast<double>(d.L);
    o.mx = mx;
    o.my = my;
    o.m2 = mx * mx + my * my;
    o.ex = ex;
    o.sx = sx;
    o.ey = ey;
    o.sy = sy;
    o.energy_per_site = -(x2 + x4) * d.inv_n;
    o.upsilon = ex - beta * n * sx * sx;  // Eq. (4), J = 1, T = 1/beta
    o.beta = beta;
    o.sweep = t;
    o.chik = sq * (0.5 * d.inv_n);  // 0 unless the lattice measures xi
    o.flipped = static_cast<uint64_t>(nf);
    d.rec[rec_count % d.rec_cap] = o;
    st->rec_count = rec_count + 1;
  }
  return o;
}

// Block 0 of a K1 launch with kCtlDraw (single lattice, fixed beta): the
// work of k_finalize, moved off the sweep's critical path, in two parts that
// run at once.  Warp kRecWarps draws the next sweep's axis and writes its
// parameters into p[par ^ 1].  With kCtlRecord, warps 0 .. kRecWarps-1
// reduce the accumulator slots that K4 of the previous sweep filled (K4 of
// this sweep refills them only after this grid completes) and append that
// sweep's record.  At fixed beta the previous sweep is t - 1 at this sweep's
// beta, so the record reads only p[par], and the two parts share no data.
// `part` is shared memory for kRecWarps x 16 int64.
constexpr int kRecWarps = 4;

__device__ __forceinline__ void k1_fold(const LatDesc &d, uint32_t ctl, long long *part) {
  DevState *st = d.st;
  const uint32_t par = ctl & kCtlPar;
  const SweepParams &now = st->p[par];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == kRecWarps) {
    if (lane == 0) {
      const uint32_t quant = st->quant, t1 = now.t + 1u;
      set_sweep_params(&st->p[par ^ 1u], quant, t1, now.cur ^ 1u, now.beta,
                       draw_axis(quant, t1, d.key0, d.key1, d.L));
    }
  } else if (warp < kRecWarps && (ctl & kCtlRecord)) {
    constexpr int kRecThreads = kRecWarps * 32;
    static_assert(kSlots * kAccStride % kRecThreads == 0 && kRecThreads % kAccStride == 0,
                  "thread i reads entries i, i + kRecThreads, ...: all of entry i % 16");
    constexpr int kPer = kSlots * kAccStride / kRecThreads;
    long long v[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) v[j] = __ldcg(d.acc + j * kRecThreads + threadIdx.x);
#pragma unroll
    for (int j = 0; j < kPer; ++j) __stcg(d.acc + j * kRecThreads + threadIdx.x, 0ll);
    long long s = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) s += v[j];
    s += __shfl_xor_sync(0xFFFFFFFFu, s, 16);
    if (lane < 16) part[warp * 16 + lane] = s;
    // named barrier 1 over the reducing warps only (the drawing warp runs on)
    asm volatile("bar.sync 1, %0;" ::"n"(kRecThreads) : "memory");
    if (warp == 0) {
      long long tot = 0;
#pragma unroll
      for (int w = 0; w < kRecWarps; ++w) tot += part[w * 16 + (lane & 15)];
      append_record(d, st, tot, now.beta, now.t - 1u, st->rec_count);
    }
  }
}

// ---------------------------------------------------------------------------
// K1: projection + bonds + coins + tile labels
// ---------------------------------------------------------------------------
// CTAs per SM: the whole-tile sweep kernels fit 6 (40 registers).  With
// FP32 thresholds 8 bytes spill, and 6 beats 5 CTAs/SM by 4.5 us and 4 by
// ~12 us at L = 4096.  In exact mode the spills (84 bytes) sit mostly on the
// rare FP64 path, and 6 CTAs/SM still beat 4 by 12.8 us per sweep.  The
// general instantiations keep 4.
template <int TY, bool EXACT, bool FROM_PLANES, bool FULL>
constexpr int k1_min_blocks() {
  return (FULL && !FROM_PLANES && TY <= 64) ? 6 : 4;
}

// ONE: the launch covers a single lattice whose descriptor is the kernel
// parameter `one` (uniform constant-bank operands, the Philox key among
// them, instead of per-thread loads of the descriptor table); otherwise
// `one` is unused and each tile finds its lattice in `descs`.  `ctl` holds
// the kCtl* bits (single lattice only; 0 for a table of lattices).
template <int TY, typename AT, bool EXACT, bool FROM_PLANES, bool FULL = false, bool ONE = false>
__global__ void __launch_bounds__(kThreads, (k1_min_blocks<TY, EXACT, FROM_PLANES, FULL>()))
    k_bond_label(const LatDesc *__restrict__ descs,
                 const uint32_t *__restrict__ prefix, uint32_t nrep,
                 uint32_t nwork, uint32_t ctl, const __grid_constant__ LatDesc one) {
  pdl_prologue_last();
  constexpr int B = TY / kWarps;  // rows per band
  extern __shared__ __align__(16) unsigned char smem[];
  // kCtlDraw: block 0 folds the finalize step, tiles start at block 1
  const uint32_t aux = (ONE && (ctl & kCtlDraw)) ? 1u : 0u;
  if (aux && blockIdx.x == 0) {
    k1_fold(one, ctl, reinterpret_cast<long long *>(smem));
    return;
  }
  uint32_t *par = reinterpret_cast<uint32_t *>(smem);
  uint32_t *sR = par + TY * 32;
  uint32_t *sD = sR + TY;
  constexpr int CAP = pair_cap<TY>();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t *pairs = sD + TY + warp * CAP;
  uint32_t *runmin = sD + TY + kWarps * CAP + warp * 32;
  runmin[lane] = kNoRoot;
  __syncwarp();

  for (uint32_t work = blockIdx.x - aux; work < nwork; work += gridDim.x - aux) {
    const uint32_t rep = ONE ? 0u : find_rep(prefix, nrep, work);
    const LatDesc &d = ONE ? one : descs[rep];
    const uint32_t tile = ONE ? work : work - __ldg(prefix + rep);
    const uint32_t L = d.L;
    const Tile g = tile_geom<TY, FULL>(L, d.ntx, d.ntx_magic, tile);
    DevState *st = d.st;
    const SweepParams &sp = st->p[ctl & kCtlPar];
    uint32_t npairs = 0u;
    const uint32_t r0 = static_cast<uint32_t>(warp) * B;
    const uint32_t nb = r0 < g.h ? min(static_cast<uint32_t>(B), g.h - r0) : 0u;
    const bool col_ok = lane < static_cast<int>(g.w);
    const uint32_t rmask = (g.w >= 32u) ? 0x7FFFFFFFu : ((1u << (g.w - 1u)) - 1u);
    const uint64_t tbase = static_cast<uint64_t>(tile) * TY;

    if (threadIdx.x == 0) d.link_count[tile] = 0u;  // the merge appends from 0
    uint32_t lab_prev = kNoRoot, D_prev = 0u;
    uint32_t labs[B];
    if (!FROM_PLANES) {
      const uint32_t t = sp.t;
      const AT *th = static_cast<const AT *>(d.theta[sp.cur]);
      const float cphi = sp.cphi32, sphi = sp.sphi32;
      const float b2 = sp.beta2_32, eps = sp.eps;
      // angles of the band, of the row below it, and (lane k < nb) of row k
      // of the column right of the tile; all loads issued up front
      float tv[B + 1];
#pragma unroll
      for (int k = 0; k <= B; ++k) {
        tv[k] = 0.0f;
        if (static_cast<uint32_t>(k) <= nb && col_ok) {
          const uint32_t r = r0 + k;
          const uint64_t row = static_cast<uint64_t>(r < g.h ? g.y0 + r : g.yh) * L;
          tv[k] = load_angle(th, row + g.x0 + lane);
        }
      }
      float tc = 0.0f;
      if (static_cast<uint32_t>(lane) < nb)
        tc = load_angle(th, static_cast<uint64_t>(g.y0 + r0 + lane) * L + g.xh);
      float a[B + 1];
#pragma unroll
      for (int k = 0; k <= B; ++k) a[k] = project32(angle_f32<AT>(tv[k]), cphi, sphi);
      const float ac = project32(angle_f32<AT>(tc), cphi, sphi);

      // phase A: bonds and coins of every row of the band (rows are
      // independent here, so their Philox chains overlap).  One BOND draw
      // serves the rows 2m and 2m + 1 of a column (counter m L + x): the
      // band starts on an even row, so row k uses words 0 and 1 of the draw
      // made at k for even k, words 2 and 3 of that draw for odd k.
      uint32_t Rws[B], Dws[B], Cws[B];
      uint32_t amb = 0u;  // exact mode: bit 2k (2k + 1) = right (down) bond of row k in the band
      Words4 rn = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int k = 0; k < B; ++k) {
        Rws[k] = Dws[k] = Cws[k] = 0u;
        if (static_cast<uint32_t>(k) >= nb) continue;  // warp-uniform
        const uint32_t r = r0 + k;
        const uint32_t gy = g.y0 + r;
        const float a_c = __shfl_sync(0xFFFFFFFFu, ac, k);
        float a_r = __shfl_down_sync(0xFFFFFFFFu, a[k], 1);
        if (static_cast<uint32_t>(lane) + 1u == g.w) a_r = a_c;
        bool br = false, bd = false, cn = false;
        if (col_ok) {
          if ((k & 1) == 0)
            rn = philox4x32_10((gy >> 1) * L + g.x0 + lane, 0u, t, kDomBond, d.key0, d.key1);
          const uint32_t w_r = (k & 1) ? rn.w2 : rn.w0, w_d = (k & 1) ? rn.w3 : rn.w1;
          // uniforms from the top 23 bits without an int->float conversion:
          // 1.m - (1 - 2^-24) is exact and is the centre of the word's 2^-23
          // bin, i.e. within 2^-24 of the FP64 uniform ((w >> 1) + 1/2) 2^-31
          const float u0 = __uint_as_float(0x3F800000u | (w_r >> 9)) - 0.99999994f;
          const float u1 = __uint_as_float(0x3F800000u | (w_d >> 9)) - 0.99999994f;
          const float xr = a[k] * a_r;
          const float xd = a[k] * a[k + 1];
          const float pr = xr > 0.0f ? 1.0f - __expf(-b2 * xr) : 0.0f;
          const float pd = xd > 0.0f ? 1.0f - __expf(-b2 * xd) : 0.0f;
          br = u0 < pr;
          bd = u1 < pd;
          if (EXACT) {
            // inside the band the FP32 decision may be wrong: settled below
            amb |= (fabsf(u0 - pr) <= eps ? 1u : 0u) << (2 * k);
            amb |= (fabsf(u1 - pd) <= eps ? 2u : 0u) << (2 * k);
          }
          cn = (w_r & 1u) != 0u;  // the coin: bit 0 of the right-bond word
        }
        Rws[k] = __ballot_sync(0xFFFFFFFFu, br);
        Dws[k] = __ballot_sync(0xFFFFFFFFu, bd);
        Cws[k] = __ballot_sync(0xFFFFFFFFu, cn);
      }
      // exact mode: the bonds inside the FP32 error band (~3e-5 of them),
      // recomputed in FP64 with the oracle's operation order.  Kept out of
      // the loop above, whose registers it would otherwise crowd; the row's
      // Philox draw is made again and the right neighbour's angle reloaded.
      if (EXACT && __any_sync(0xFFFFFFFFu, amb != 0u)) {
#pragma unroll
        for (int k = 0; k < B; ++k) {
          const uint32_t m2 = (amb >> (2 * k)) & 3u;
          if (!__any_sync(0xFFFFFFFFu, m2 != 0u)) continue;
          bool br = (Rws[k] >> lane) & 1u, bd = (Dws[k] >> lane) & 1u;
          if (m2) {
            const uint32_t gy = g.y0 + r0 + k;
            const Words4 w =
                philox4x32_10((gy >> 1) * L + g.x0 + lane, 0u, t, kDomBond, d.key0, d.key1);
            if (m2 & 1u) {
              const float th_r =
                  (static_cast<uint32_t>(lane) + 1u == g.w)
                      ? load_angle(th, static_cast<uint64_t>(gy) * L + g.xh)
                      : load_angle(th, static_cast<uint64_t>(gy) * L + g.x0 + lane + 1u);
              const bool e = bond_fp64(angle_f64<AT>(tv[k]), angle_f64<AT>(th_r),
                                       (k & 1) ? w.w2 : w.w0, sp.beta, sp.cphi, sp.sphi);
              atomicAdd(&st->n_fp64, 1ull);
              if (e != br) atomicAdd(&st->n_fp32_wrong, 1ull);
              br = e;
            }
            if (m2 & 2u) {
              const bool e = bond_fp64(angle_f64<AT>(tv[k]), angle_f64<AT>(tv[k + 1]),
                                       (k & 1) ? w.w3 : w.w1, sp.beta, sp.cphi, sp.sphi);
              atomicAdd(&st->n_fp64, 1ull);
              if (e != bd) atomicAdd(&st->n_fp32_wrong, 1ull);
              bd = e;
            }
          }
          Rws[k] = __ballot_sync(0xFFFFFFFFu, br);
          Dws[k] = __ballot_sync(0xFFFFFFFFu, bd);
        }
      }
      // one store per plane for the whole band: lane k writes row r0 + k
      {
        uint32_t Rw = 0u, Dw = 0u, Cw = 0u;
#pragma unroll
        for (int k = 0; k < B; ++k) {
          if (lane == k) {
            Rw = Rws[k];
            Dw = Dws[k];
            Cw = Cws[k];
          }
        }
        if (static_cast<uint32_t>(lane) < nb) {
          const uint32_t r = r0 + lane;
          d.rplane[tbase + r] = Rw;
          d.dplane[tbase + r] = Dw;
          sR[r] = Rw;
          sD[r] = Dw;
          const uint32_t i0 = (g.y0 + r) * L + g.x0;
          if (FULL || !d.ragged) {
            d.coin[i0 >> 5] = Cw;
          } else if (Cw) {
            const uint32_t off = i0 & 31u;
            atomicOr(d.coin + (i0 >> 5), Cw << off);
            if (off) atomicOr(d.coin + (i0 >> 5) + 1, Cw >> (32u - off));
          }
        }
      }
      // phase B: the row scan of the band
#pragma unroll
      for (int k = 0; k < B; ++k) {
        if (static_cast<uint32_t>(k) >= nb) break;
        const uint32_t up = (k > 0 && ((D_prev >> lane) & 1u)) ? lab_prev : kNoRoot;
        lab_prev = scan_row<CAP>(par, pairs, npairs, runmin, r0 + k, ~((Rws[k] & rmask) << 1), up, lane);
        labs[k] = lab_prev;
        D_prev = Dws[k];
      }
    } else {
#pragma unroll
      for (int k = 0; k < B; ++k) {
        if (static_cast<uint32_t>(k) >= nb) break;
        const uint32_t r = r0 + k;
        const uint32_t Rw = __ldg(d.rplane + tbase + r);
        const uint32_t Dw = __ldg(d.dplane + tbase + r);
        if (lane == 0) {
          sR[r] = Rw;
          sD[r] = Dw;
        }
        const uint32_t up = (k > 0 && ((D_prev >> lane) & 1u)) ? lab_prev : kNoRoot;
        lab_prev = scan_row<CAP>(par, pairs, npairs, runmin, r, ~((Rw & rmask) << 1), up, lane);
        labs[k] = lab_prev;
        D_prev = Dw;
      }
    }
    __syncthreads();
    // all threads at once: the warp's recorded equivalences, and the join of
    // each band to the one above it across their boundary rows
    const uint32_t np = min(npairs, static_cast<uint32_t>(CAP));
    for (uint32_t e = lane; e < np; e += 32u) {
      const uint32_t pr = pairs[e];
      sunion(par, pr >> 16, pr & 0xFFFFu);
    }
    if (warp > 0 && nb > 0) {
      const uint32_t r = r0 - 1u;
      const uint32_t D = sD[r];
      const uint32_t Ra = sR[r] & rmask, Rb = sR[r0] & rmask;
      const uint32_t V = D & ~((D & Ra & Rb) << 1);
      if (col_ok && ((V >> lane) & 1u))
        sunion(par, r * 32u + run_start_of(~(Ra << 1), lane),
               r0 * 32u + run_start_of(~(Rb << 1), lane));
    }
    __syncthreads();
    // every site: root of its run's root as recorded by the scan; boundary
    // sites also into the tile's edge table
    uint32_t *edge = d.edge + static_cast<uint64_t>(tile) * edge_words<TY>();
#pragma unroll
    for (int k = 0; k < B; ++k) {
      if (static_cast<uint32_t>(k) >= nb) break;
      const uint32_t r = r0 + k;
      if (col_ok) {
        const uint32_t root = sfind2(par, labs[k]);
        const uint32_t v = (g.y0 + (root >> 5)) * L + g.x0 + (root & 31u);
        d.label[static_cast<uint64_t>(g.y0 + r) * L + g.x0 + lane] = v;
        if (lane == 0) edge[r] = v;                                      // left column
        if (static_cast<uint32_t>(lane) + 1u == g.w) edge[TY + r] = v;  // right column
        if (r == 0u) edge[2 * TY + lane] = v;                           // top row
        if (r + 1u == g.h) edge[2 * TY + 32 + lane] = v;                // bottom row
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// K2: merge across tile edges.  Work item = (tile, j): j < TY is the right
// edge of tile row j, j >= TY the bottom edge of column j - TY.
// ---------------------------------------------------------------------------
// Edge item j of a tile: j < TY is the bond from row j of its right column
// to the next tile, j >= TY the bond from column j - TY of its bottom row to
// the tile below.  Returns whether that bond exists and is active, and the
// tile roots of its two endpoints from the edge table.  The roots are loaded
// together with the bond's plane word (all three addresses lie inside their
// arrays whatever the bond), so the chain of dependent loads is one shorter.
// (Repeated unions of the same two tile roots are grouped in k_merge; a
// check of the neighbouring bonds here saved fewer of them than its plane
// loads cost.)
template <int TY, bool FULL>
__device__ __forceinline__ bool edge_roots(const LatDesc &d, uint32_t tile, uint32_t j,
                                           uint32_t *ta, uint32_t *tb) {
  constexpr uint32_t EW = edge_words<TY>();
  const Tile g = tile_geom<TY, FULL>(d.L, d.ntx, d.ntx_magic, tile);
  const uint64_t base = static_cast<uint64_t>(tile) * TY;
  const uint32_t tx = g.x0 >> 5;
  const uint32_t *plane;
  uint64_t ea, eb;
  uint32_t bit;
  bool valid;
  if (j < static_cast<uint32_t>(TY)) {
    // the neighbouring tile to the right holds column xh as its column 0
    const uint32_t tn = tile - tx + (tx + 1u == d.ntx ? 0u : tx + 1u);
    valid = j < g.h;
    bit = g.w - 1u;
    plane = d.rplane + base + j;
    ea = static_cast<uint64_t>(tile) * EW + TY + j;  // right column, row j
    eb = static_cast<uint64_t>(tn) * EW + j;         // its left column, row j
  } else {
    // the tile below holds row yh as its row 0, same columns
    const uint32_t c = j - TY;
    const uint32_t ty = g.y0 / static_cast<uint32_t>(TY);
    const uint32_t tb_ = (ty + 1u == d.nty ? 0u : (ty + 1u) * d.ntx) + tx;
    valid = c < g.w;
    bit = c;
    plane = d.dplane + base + g.h - 1u;
    ea = static_cast<uint64_t>(tile) * EW + 2 * TY + 32 + c;  // bottom row, column c
    eb = static_cast<uint64_t>(tb_) * EW + 2 * TY + c;        // its top row, column c
  }
  const uint32_t w = __ldg(plane);
  *ta = __ldg(d.edge + ea);
  *tb = __ldg(d.edge + eb);
  return valid && ((w >> bit) & 1u);
}

// The edge items of one warp (a tile edge, or parts of two for TY = 16 and
// 128) whose endpoints have the same pair of tile roots would repeat the same
// union; __match_any_sync on the pair (and on the lattice, as root indices
// are per lattice) lets one lane of each group do it (merge at L = 4096:
// 34.3 -> 29.0 us).  Lanes past the last item stay in the warp, clamped and
// inactive, so every match sees all 32.
struct EdgeItem {
  const LatDesc *d;
  uint32_t rep, tile, ta, tb;
  bool act;
};

template <int TY, bool FULL, bool ONE>
__device__ __forceinline__ EdgeItem edge_item(const LatDesc *__restrict__ descs,
                                              const uint32_t *__restrict__ prefix,
                                              uint32_t nrep, uint32_t nwork, uint64_t item,
                                              const LatDesc &one) {
  const uint64_t per = TY + 32;
  const uint64_t total = static_cast<uint64_t>(nwork) * per;  // > 0: launches have work
  const uint64_t it = item < total ? item : total - 1u;
  const uint32_t work = static_cast<uint32_t>(it / per);
  const uint32_t j = static_cast<uint32_t>(it % per);
  EdgeItem e;
  e.rep = ONE ? 0u : find_rep(prefix, nrep, work);
  e.d = ONE ? &one : descs + e.rep;
  const uint32_t tile = ONE ? work : work - __ldg(prefix + e.rep);
  e.tile = tile;
  const bool bond = edge_roots<TY, FULL>(*e.d, tile, j, &e.ta, &e.tb);
  e.act = item < total && bond;
  if (!e.act) e.ta = e.tb = 0u;
  return e;
}

// true on the lowest lane of each group of lanes holding the same key (and
// lattice: ONE launches have only one)
template <bool ONE>
__device__ __forceinline__ bool group_leader(unsigned long long key, uint32_t rep) {
  unsigned m = __match_any_sync(0xFFFFFFFFu, key);
  if (!ONE) m &= __match_any_sync(0xFFFFFFFFu, rep);
  return (threadIdx.x & 31u) == static_cast<unsigned>(__ffs(m) - 1);
}

// One thread per edge item; the loop over batches of 32 items (warp w of
// the grid takes batches w, w + W, ...) lets any grid size cover the items.
// ONE: a single lattice whose descriptor is the parameter `one`, as in K1.
template <int TY, bool FULL = false, bool ONE = false>
__global__ void __launch_bounds__(kThreads)
    k_merge(const LatDesc *__restrict__ descs,
            const uint32_t *__restrict__ prefix, uint32_t nrep,
            uint32_t nwork, const __grid_constant__ LatDesc one) {
  pdl_prologue();
  if (nwork == 0u) return;
  const uint64_t total = static_cast<uint64_t>(nwork) * (TY + 32);
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kThreads;
  // start from the tile roots (from the edge table): labels of non-root sites
  // are never written here, so after the merge every site still points at
  // its tile root
  for (uint64_t base = static_cast<uint64_t>(blockIdx.x) * kThreads + (threadIdx.x & ~31u);
       base < total; base += stride) {
    const EdgeItem e =
        edge_item<TY, FULL, ONE>(descs, prefix, nrep, nwork, base + (threadIdx.x & 31u), one);
    const unsigned long long key =
        e.act ? (static_cast<unsigned long long>(e.ta) << 32 | e.tb) : ~0ull;
    if (group_leader<ONE>(key, e.rep) && e.act)
      gunion(e.d->label, static_cast<uint64_t>(e.d->L) * e.d->L, e.ta, e.tb, e.d->st, e.d->find_cap,
             e.d->links + static_cast<uint64_t>(e.tile) * (TY + 32u), e.d->link_count + e.tile,
             min(e.d->link_cap, TY + 32u));
  }
}

// Pointer jumping: x re-points at its grandparent until its parent is a
// root.  When all linked roots jump concurrently, a chain of length d
// collapses in O(log d) steps per node instead of a walk of length d.  Only
// ancestors are ever written and roots no longer change.
__device__ __forceinline__ void jump(uint32_t *lab, uint64_t n, uint32_t x, DevState *st,
                                     uint32_t cap) {
  x = chk(x, n, st);
  for (uint32_t it = 0; it < cap; ++it) {
    const uint32_t p = chk(__ldcg(lab + x), n, st);
    if (p == x) return;
    const uint32_t gp = chk(__ldcg(lab + p), n, st);
    if (gp == p) return;
    __stcg(lab + x, gp);
  }
  atomicOr(&st->err, kErrFindCap);
}

// K3: every root the merge linked jumps (concurrently with the others) until
// its parent is a root.  Every entry the merge changed is such a root's: the
// link itself, or path halving, which only re-points nodes that already have
// a parent.  Thread j of a tile's edge items takes the tile's j-th link.
// One warp per tile (k_compress CTA b holds tiles 8b .. 8b + 7): its lanes
// take the tile's links j = lane, lane + 32, ... below the tile's count, so
// tiles that linked nothing cost one load.
template <int TY, bool ONE = false>
__global__ void __launch_bounds__(kThreads)
    k_compress(const LatDesc *__restrict__ descs,
               const uint32_t *__restrict__ prefix, uint32_t nrep,
               uint32_t nwork, const __grid_constant__ LatDesc one) {
  pdl_prologue();
  const uint32_t work = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (work >= nwork) return;
  const uint32_t rep = ONE ? 0u : find_rep(prefix, nrep, work);
  const LatDesc &d = ONE ? one : descs[rep];
  const uint32_t tile = ONE ? work : work - __ldg(prefix + rep);
  constexpr uint32_t per = TY + 32;
  const uint32_t count = min(__ldcg(d.link_count + tile), min(d.link_cap, per));
  const uint32_t *links = d.links + static_cast<uint64_t>(tile) * per;
  const uint64_t n = static_cast<uint64_t>(d.L) * d.L;
  for (uint32_t j = threadIdx.x & 31u; j < count; j += 32u)
    jump(d.label, n, __ldcg(links + j), d.st, d.find_cap);
}

// CTAs of k_compress for nwork tiles
inline uint32_t compress_blocks(uint32_t nwork) { return (nwork + kWarps - 1) / kWarps; }

// ---------------------------------------------------------------------------
// K4: canonical labels, flip, observable sums
// ---------------------------------------------------------------------------
// Fixed point of a term v in [-1, 1]: v + 3 lies in [2, 4], whose FP32 grid
// step is 2^-22, so the bit pattern of v + 3 minus that of 3.0 (0x40400000)
// is round(v * 2^22).  The kernels sum the patterns and take the constant off
// per summed term afterwards.
__device__ __forceinline__ uint32_t fix22_bits(float v) {
  return __float_as_uint(__fadd_rn(v, 3.0f));
}

template <int TY>
constexpr size_t flip_smem() {
  return 0;
}

// K4 layout: as K1, warp w owns rows r0 .. r0+B-1 of the tile (lane =
// column) and also resolves the row below its band (the next band's first
// row, or the row below the tile) and, with lanes 0..B-1, the column right of
// the tile.  Roots come in two batched rounds of loads: a site's entry (its
// tile root, or its root where this kernel already rewrote it), then that
// entry's entry,
// which k_compress has made the root (every merged tile root is jumped until
// its parent is a root; an unmerged one is its own entry).
// EXT: the extended instantiation, for lattice tables where some lattice
// measures chik (d.xi) or runs Wolff updates (d.wolff); each lattice still
// takes only what its own flags ask for.  The lean one does neither and
// keeps its registers (launch bounds 5 CTAs/SM; EXT needs 4).
// WL: also store the canonical labels (for a sweep whose labels the host may
// read back, and always with LABELS_ONLY); otherwise the next sweep's K1
// overwrites them, and leaving the store out saves ~8 us per sweep at
// L = 4096.
template <int TY, typename AT, bool LABELS_ONLY, bool EXT = false, bool WL = true,
          bool FULL = false, bool ONE = false>
__global__ void __launch_bounds__(kThreads, EXT ? 4 : 5)
    k_flip_measure(const LatDesc *__restrict__ descs,
                   const uint32_t *__restrict__ prefix, uint32_t nrep,
                   uint32_t nwork, uint32_t par, const __grid_constant__ LatDesc one) {
  pdl_prologue_last();
  constexpr int B = TY / kWarps;
  __shared__ long long red[kWarps][EXT ? 15 : 6];  // EXT: 14 sums + flip count
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (uint32_t work = blockIdx.x; work < nwork; work += gridDim.x) {
    const uint32_t rep = ONE ? 0u : find_rep(prefix, nrep, work);
    const LatDesc &d = ONE ? one : descs[rep];
    const uint32_t tile = ONE ? work : work - __ldg(prefix + rep);
    const uint32_t L = d.L;
    const Tile g = tile_geom<TY, FULL>(L, d.ntx, d.ntx_magic, tile);
    DevState *st = d.st;
    const SweepParams &sp = st->p[par];  // par: the sweep's parameter slot
    const uint32_t cur = sp.cur;
    const float c32 = sp.c32;
    const AT *thin = static_cast<const AT *>(d.theta[cur]);
    AT *thout = static_cast<AT *>(d.theta[cur ^ 1u]);
    uint32_t *lab = d.label;
    const uint32_t r0 = static_cast<uint32_t>(warp) * B;
    const uint32_t nb = r0 < g.h ? min(static_cast<uint32_t>(B), g.h - r0) : 0u;
    const bool col_ok = lane < static_cast<int>(g.w);
    const bool vc = static_cast<uint32_t>(lane) < nb;  // column xh, row r0+lane
    const uint64_t ic = static_cast<uint64_t>(g.y0 + r0 + lane) * L + g.xh;

    // step 1: labels and angles of rows r0 .. r0+nb and of column xh
    uint32_t l[B + 1];
    float t[B + 1];
#pragma unroll
    for (int k = 0; k <= B; ++k) {
      l[k] = 0u;
      t[k] = 0.0f;
      if (static_cast<uint32_t>(k) <= nb && col_ok) {
        const uint32_t r = r0 + k;
        const uint64_t i = static_cast<uint64_t>(r < g.h ? g.y0 + r : g.yh) * L + g.x0 + lane;
        l[k] = __ldcg(lab + i);
        if (!LABELS_ONLY) t[k] = load_angle(thin, i);
      }
    }
    uint32_t lc = 0u;
    float tc = 0.0f;
    if (vc) {
      lc = __ldcg(lab + ic);
      if (!LABELS_ONLY) tc = load_angle(thin, ic);
    }
    // step 2: the tile root's entry
    const uint64_t nsites = static_cast<uint64_t>(L) * L;
    uint32_t p[B + 1];
#pragma unroll
    for (int k = 0; k <= B; ++k)
      p[k] = (static_cast<uint32_t>(k) <= nb && col_ok) ? chk(__ldcg(lab + chk(l[k], nsites, st)), nsites, st) : 0u;
    const uint32_t pc = vc ? chk(__ldcg(lab + chk(lc, nsites, st)), nsites, st) : 0u;
    // after k_compress a site's entry is its tile root or its root, and a
    // tile root's entry is itself or its root: the entry's entry is the root
#pragma unroll
    for (int k = 0; k <= B; ++k)
      if (static_cast<uint32_t>(k) <= nb && col_ok) l[k] = p[k];
    if (vc) lc = pc;
    // canonical labels of the band's own sites
    if constexpr (LABELS_ONLY || WL) {
#pragma unroll
      for (int k = 0; k < B; ++k) {
        if (static_cast<uint32_t>(k) < nb && col_ok)
          __stcg(lab + static_cast<uint64_t>(g.y0 + r0 + k) * L + g.x0 + lane, l[k]);
      }
    }
    if (LABELS_ONLY) continue;
    // step 3: which sites reflect.  SW: the coin of the site's root.
    // Wolff: the sites of the seed site's cluster, whose root is the entry's
    // entry of the seed like any other site's (whether or not this kernel
    // has already rewritten those entries: both reads give the root)
    uint32_t f[B + 1], fc;
    int nflip = 0;  // Wolff: reflected sites of the band (warp-uniform)
    if (EXT && d.wolff) {
      const uint32_t r0 = __ldcg(lab + chk(__ldcg(lab + sp.seed_site), nsites, st));
#pragma unroll
      for (int k = 0; k <= B; ++k)
        f[k] = (static_cast<uint32_t>(k) <= nb && col_ok && l[k] == r0) ? 1u : 0u;
      fc = (vc && lc == r0) ? 1u : 0u;
#pragma unroll
      for (int k = 0; k < B; ++k)
        nflip += __popc(__ballot_sync(0xFFFFFFFFu, f[k] && static_cast<uint32_t>(k) < nb));
    } else {
#pragma unroll
      for (int k = 0; k <= B; ++k)
        f[k] = (static_cast<uint32_t>(k) <= nb && col_ok)
                   ? (__ldg(d.coin + (l[k] >> 5)) >> (l[k] & 31u)) & 1u
                   : 0u;
      fc = vc ? (__ldg(d.coin + (lc >> 5)) >> (lc & 31u)) & 1u : 0u;
    }
    // reflection, stores, and cos/sin of the new angles
    float co[B + 1], sn[B + 1];
#pragma unroll
    for (int k = 0; k <= B; ++k) {
      float nv = t[k];
      if (f[k]) {
        nv = reflect<AT>(t[k], c32);
        if (static_cast<uint32_t>(k) < nb && col_ok)
          thout[static_cast<uint64_t>(g.y0 + r0 + k) * L + g.x0 + lane] = store_exact<AT>(nv);
      } else if (static_cast<uint32_t>(k) < nb && col_ok) {
        thout[static_cast<uint64_t>(g.y0 + r0 + k) * L + g.x0 + lane] = store_exact<AT>(t[k]);
      }
      sin_cos<AT>(nv, &sn[k], &co[k]);
    }
    float cc, sc;
    sin_cos<AT>(fc ? reflect<AT>(tc, c32) : tc, &sc, &cc);
    // observable terms of the band's own sites (with d.xi also the Fourier
    // sums of chik: s(r) times (cos, sin)(2 pi x / L) and (2 pi y / L))
    // Each term's fixed-point value is the bit pattern of v + 3 minus that of
    // 3.0 (fix22); the patterns are summed modulo 2^32 and the constant is
    // taken off once per thread below (exact: the true sum fits in 32 bits).
    constexpr int NV = EXT ? 14 : 6;
    uint32_t acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0u;
    const bool xi = EXT && d.xi != 0u;
    float2 wx = make_float2(0.0f, 0.0f);
    if constexpr (EXT) {
      if (xi && col_ok) wx = __ldg(d.wave + g.x0 + lane);
    }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      if (static_cast<uint32_t>(k) >= nb) break;  // warp-uniform
      const float cxh = __shfl_sync(0xFFFFFFFFu, cc, k);
      const float sxh = __shfl_sync(0xFFFFFFFFu, sc, k);
      float cr = __shfl_down_sync(0xFFFFFFFFu, co[k], 1);
      float sr = __shfl_down_sync(0xFFFFFFFFu, sn[k], 1);
      if (static_cast<uint32_t>(lane) + 1u == g.w) {
        cr = cxh;
        sr = sxh;
      }
      if (col_ok) {
        const float ci = co[k], si = sn[k], cd = co[k + 1], sd = sn[k + 1];
        acc[0] += fix22_bits(ci);
        acc[1] += fix22_bits(si);
        acc[2] += fix22_bits(fmaf(ci, cr, si * sr));
        acc[3] += fix22_bits(fmaf(si, cr, -(ci * sr)));
        acc[4] += fix22_bits(fmaf(ci, cd, si * sd));
        acc[5] += fix22_bits(fmaf(si, cd, -(ci * sd)));
        if constexpr (EXT) {
          if (xi) {
            const float2 wy = __ldg(d.wave + g.y0 + r0 + k);
            acc[NV - 8] += fix22_bits(ci * wx.x);
            acc[NV - 7] += fix22_bits(ci * wx.y);
            acc[NV - 6] += fix22_bits(si * wx.x);
            acc[NV - 5] += fix22_bits(si * wx.y);
            acc[NV - 4] += fix22_bits(ci * wy.x);
            acc[NV - 3] += fix22_bits(ci * wy.y);
            acc[NV - 2] += fix22_bits(si * wy.x);
            acc[NV - 1] += fix22_bits(si * wy.y);
          }
        }
      }
    }
    const int nv = xi ? 14 : 6;
    // rows this thread summed: the offset of 3.0 comes off once per row
    const uint32_t rows = col_ok ? nb : 0u;
    long long v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const int t = static_cast<int>(acc[k] - rows * 0x40400000u);  // |sum| <= B 2^22
      if constexpr (B <= 8) {
        // a warp's sum stays within 32 x 8 x 2^22 = 2^30: one 32-bit warp
        // reduction instruction (exact integer sum)
        v[k] = (k < nv) ? __reduce_add_sync(0xFFFFFFFFu, t) : t;
      } else {
        v[k] = t;
        if (k < nv) {
#pragma unroll
          for (int off = 16; off > 0; off >>= 1)
            v[k] += __shfl_down_sync(0xFFFFFFFFu, v[k], off);
        }
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) red[warp][k] = v[k];
      if constexpr (EXT) red[warp][NV] = nflip;
    }
    __syncthreads();
    if (threadIdx.x < static_cast<unsigned>(nv)) {
      long long sum = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) sum += red[w][threadIdx.x];
      atomicAdd(reinterpret_cast<unsigned long long *>(
                    d.acc + (tile % kSlots) * kAccStride + threadIdx.x),
                static_cast<unsigned long long>(sum));
    }
    if constexpr (EXT) {
      if (threadIdx.x == 32u && d.wolff) {
        long long sum = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) sum += red[w][NV];
        atomicAdd(reinterpret_cast<unsigned long long *>(
                      d.acc + (tile % kSlots) * kAccStride + kFlipSlot),
                  static_cast<unsigned long long>(sum));
      }
    }
    __syncthreads();
  }
}

// K5: one CTA of two warps per lattice.  Warp 0 reduces the accumulator
// slots and derives the record and the PCC step; warp 1 meanwhile draws the
// axis of the next sweep, so the two FP64 chains run on two schedulers at
// once.  Lane k of warp 0 ends with the sum of entry k over all slots: one
// FP64 instruction then converts (and one scales) all of them, instead of a
// serial chain on one lane.  mode 0: the full step, the next parameters in
// both slots; mode kFinRecord | par: the last record of a fixed-beta call
// (see kCtlDraw), no axis to draw.
constexpr int kFinalizeThreads = 64;

static __global__ void __launch_bounds__(kFinalizeThreads)
    k_finalize(const LatDesc *__restrict__ descs, uint32_t nrep, uint32_t mode) {
  const uint32_t rep = blockIdx.x;
  if (rep >= nrep) return;
  // The kernel is a chain of dependent memory accesses (ncu: ~11 us for
  // under a thousand instructions when each field was loaded where it was
  // used), so everything it reads is loaded in one batch: the descriptor and
  // the state as whole structs, then the accumulator slots beside the state.
  const LatDesc d = descs[rep];  // static: loaded before the wait
  pdl_prologue();
  DevState *st = d.st;
  const DevState s0 = *st;
  const bool record_only = (mode & kFinRecord) != 0u;
  const uint32_t par = mode & kCtlPar;
  // selects, not s0.p[par]: a run-time index would put s0 in local memory
  const SweepParams sp = par ? s0.p[1] : s0.p[0];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ Axis next;
  static_assert(kSlots * kAccStride == 32 * 32 && kAccStride == 16,
                "the slots read as 32 rows of 32 entries, lane l holding entry l % 16");
  double nb = sp.beta;  // beta of the next sweep (thread 0)
  if (warp == 1) {
    if (lane == 0 && !record_only) next = draw_axis(s0.quant, sp.t + 1u, d.key0, d.key1, d.L);
  } else {
    // Row i of 32 consecutive entries holds slots 2i and 2i + 1, so lane l
    // reads entry l % 16 of slot 2i + l / 16: every load and store is
    // coalesced (lane = slot, 128 B apart, had cost ~5.6 us per sweep).
    long long v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __ldcg(d.acc + i * 32 + lane);
#pragma unroll
    for (int i = 0; i < 32; ++i) __stcg(d.acc + i * 32 + lane, 0ll);
    long long tot = 0;  // lane k and lane k + 16: entry k summed over all slots
#pragma unroll
    for (int i = 0; i < 32; ++i) tot += v[i];
    tot += __shfl_xor_sync(0xFFFFFFFFu, tot, 16);
    const ObsRecord o = append_record(d, st, tot, sp.beta, sp.t, s0.rec_count);
    if (lane == 0 && s0.pcc_on) {
      const double beta = sp.beta;
      double acc = s0.pcc_acc + beta * o.upsilon;
      uint32_t count = s0.pcc_count + 1;
      if (count >= s0.pcc_block) {
        const double mean = acc / static_cast<double>(s0.pcc_block);
        double db = s0.pcc_dbeta0;
        if (s0.pcc_halve) db = ldexp(db, -static_cast<int>(s0.pcc_k / s0.pcc_halve));
        nb = (mean < s0.pcc_target) ? beta + db : beta - db;
        acc = 0.0;
        count = 0;
      }
      st->pcc_acc = acc;
      st->pcc_count = count;
      st->pcc_k = s0.pcc_k + 1;
    }
  }
  __syncthreads();  // both warps: the next axis from warp 1
  if (threadIdx.x == 0) {
    if (record_only) {
      st->p[par] = par ? s0.p[0] : s0.p[1];
    } else {
      set_sweep_params(&st->p[0], s0.quant, sp.t + 1u, sp.cur ^ 1u, nb, next);
      st->p[1] = st->p[0];
    }
  }
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
      if constexpr (std::is_same<AT, uint16_t>::value) {
        v = static_cast<float>(w.w0 >> 16);  // q: the word's top 16 bits
      } else {
        const float step = 6.2831854820251465f * 0x1p-24f;
        v = __fmul_rn(static_cast<float>(w.w0 >> 8), step);
        if (v >= two_pi_f()) v = 0.0f;
      }
    }
    th[i] = store_value<AT>(v);
  }
}

// (cos, sin)(2 pi x / L) for the Fourier sums of chik, rounded from FP64
static __global__ void k_init_wave(LatDesc d) {
  const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= d.L) return;
  double s, c;
  sincospi(2.0 * static_cast<double>(x) / static_cast<double>(d.L), &s, &c);
  const_cast<float2 *>(d.wave)[x] = make_float2(__double2float_rn(c), __double2float_rn(s));
}

static __global__ void k_init_state(LatDesc d, double beta, uint32_t quant) {
  DevState *st = d.st;
  st->quant = quant;
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
  set_sweep_params(&st->p[0], quant, 0u, 0u, beta, draw_axis(quant, 0u, d.key0, d.key1, d.L));
  st->p[1] = st->p[0];
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
