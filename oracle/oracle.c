/*
 * oracle.c -- plain, sequential CPU oracle of the Swendsen-Wang sweep for the
 * 2D classical XY model (Wolff embedding).  TEST INFRASTRUCTURE ONLY: see
 * oracle.h for who may use it, the order of the steps and the conventions.
 *
 * Written for clarity, not speed: every step is a separate loop over the
 * lattice, in the order the method defines, with FP64 arithmetic.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* 2*pi and pi as FP64 literals, and 2*pi rounded to FP32. */
#define ORC_TWO_PI 6.283185307179586
#define ORC_PI 3.141592653589793
#define ORC_TWO_PI_F ((float)6.283185307179586)
/* u16 angle step 2pi / 65536 (a power-of-two scaling of ORC_TWO_PI: exact) */
#define ORC_U16_STEP (ORC_TWO_PI / 65536.0)

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 3): ten rounds of two 32x32->64  */
/* multiplications, a counter permutation and a key xor, with the key bumped */
/* by the Weyl constants between rounds.                                     */
/* ------------------------------------------------------------------------ */
#define PHILOX_MUL0 0xD2511F53u
#define PHILOX_MUL1 0xCD9E8D57u
#define PHILOX_WEYL0 0x9E3779B9u
#define PHILOX_WEYL1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_WEYL0;
      k1 += PHILOX_WEYL1;
    }
    uint64_t prod0 = (uint64_t)PHILOX_MUL0 * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)PHILOX_MUL1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void philox_draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                        uint32_t c3, uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

void orc_philox_stream(uint64_t seed, const uint32_t ctr[4], int word,
                       uint64_t n_calls, uint32_t *out) {
  for (uint64_t k = 0; k < n_calls; ++k) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    c[word & 3] += (uint32_t)k;
    philox_draw(seed, c[0], c[1], c[2], c[3], out + 4 * k);
  }
}

/* ------------------------------------------------------------------------ */
/* FP16 storage helpers (IEEE binary16 via the compiler's _Float16).         */
/* ------------------------------------------------------------------------ */
static float half_bits_to_float(uint16_t b) {
  _Float16 h;
  memcpy(&h, &b, 2);
  return (float)h;
}

static uint16_t float_to_half_bits(float v) {
  _Float16 h = (_Float16)v; /* round to nearest even */
  uint16_t b;
  memcpy(&b, &h, 2);
  return b;
}

/* Store an angle v in [0, 2pi_f) as FP16; a value that rounds up to 2pi or
 * beyond is wrapped once more (angles live in [0, 2pi)). */
static uint16_t store_angle_f16(float v) {
  uint16_t b = float_to_half_bits(v);
  float back = half_bits_to_float(b);
  if (back >= ORC_TWO_PI_F) b = float_to_half_bits(back - ORC_TWO_PI_F);
  return b;
}

/* Wrap an FP32 angle in (-2pi, 2pi] into [0, 2pi) with FP32 operations. */
static float wrap_f32(float v) {
  if (v < 0.0f) v = v + ORC_TWO_PI_F;
  if (v >= ORC_TWO_PI_F) v = v - ORC_TWO_PI_F;
  return v;
}

/* ------------------------------------------------------------------------ */
/* Step 1: the random axis of sweep t (Wolff's embedding).                   */
/* ------------------------------------------------------------------------ */
void orc_axis(uint64_t seed, uint32_t t, double out[4], float *c32) {
  uint32_t w[4];
  philox_draw(seed, 0u, 0u, t, ORC_DOM_AXIS, w);
  uint64_t bits = ((uint64_t)w[0] << 32) | (uint64_t)w[1];
  double u = (double)(bits >> 11) * 0x1.0p-53; /* uniform in [0, 1) */
  double phi = ORC_TWO_PI * u;
  double c = fmod(ORC_PI + 2.0 * phi, ORC_TWO_PI);
  out[0] = phi;
  out[1] = cos(phi);
  out[2] = sin(phi);
  out[3] = c;
  float cf = (float)c;
  if (cf >= ORC_TWO_PI_F) cf = 0.0f;
  *c32 = cf;
}

/* The axis of sweep t for u16 fixed-point angles, theta = q 2pi / 65536.
 * The reflection constant has to lie on the angle grid for the flip to be
 * the exact integer map q -> (Cq - q) mod 65536, and the bonds have to use
 * the axis that this map reflects about, or the flipped projection would not
 * be exactly the negated one.  So the axis is put on the grid: m = the 16
 * bits of the axis word below its top bit (phi mod pi = pi frac(2u), floored
 * to the grid), phi_q = pi m / 65536 and Cq = (m + 32768) mod 65536, so that
 * pi + 2 phi_q = Cq 2pi / 65536 (mod 2pi).  phi_q and phi_q + pi give the
 * same bonds and the same reflection. */
void orc_axis_u16(uint64_t seed, uint32_t t, double out[4], uint16_t *cq) {
  uint32_t w[4];
  philox_draw(seed, 0u, 0u, t, ORC_DOM_AXIS, w);
  uint64_t bits = ((uint64_t)w[0] << 32) | (uint64_t)w[1];
  uint32_t m = (uint32_t)(bits >> 47) & 0xFFFFu;
  double phi = ORC_PI * ((double)m / 65536.0);
  uint32_t c = (m + 32768u) & 0xFFFFu;
  out[0] = phi;
  out[1] = cos(phi);
  out[2] = sin(phi);
  out[3] = (double)c * ORC_U16_STEP;
  *cq = (uint16_t)c;
}

/* ------------------------------------------------------------------------ */
/* Initial angles.                                                           */
/* ------------------------------------------------------------------------ */
static float init_angle(uint64_t seed, uint64_t i, int start) {
  if (start != 0) return 0.0f;
  uint32_t w[4];
  philox_draw(seed, (uint32_t)i, (uint32_t)(i >> 32), 0xffffffffu,
              ORC_DOM_INIT, w);
  float step = ORC_TWO_PI_F * 0x1.0p-24f; /* exact: a power-of-two scaling */
  float v = (float)(w[0] >> 8) * step;
  if (v >= ORC_TWO_PI_F) v = 0.0f;
  return v;
}

void orc_init_angles_f32(int Lx, int Ly, uint64_t seed, int start,
                         float *theta) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  for (uint64_t i = 0; i < n; ++i) theta[i] = init_angle(seed, i, start);
}

void orc_init_angles_f16(int Lx, int Ly, uint64_t seed, int start,
                         uint16_t *theta_bits) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  for (uint64_t i = 0; i < n; ++i)
    theta_bits[i] = store_angle_f16(init_angle(seed, i, start));
}

/* u16: the top 16 bits of the same INIT word (theta = q 2pi / 65536). */
void orc_init_angles_u16(int Lx, int Ly, uint64_t seed, int start,
                         uint16_t *q) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  for (uint64_t i = 0; i < n; ++i) {
    q[i] = 0;
    if (start != 0) continue;
    uint32_t w[4];
    philox_draw(seed, (uint32_t)i, (uint32_t)(i >> 32), 0xffffffffu,
                ORC_DOM_INIT, w);
    q[i] = (uint16_t)(w[0] >> 16);
  }
}

/* ------------------------------------------------------------------------ */
/* Lattice neighbours.  Returns 0 if the link does not exist (open edge).    */
/* ------------------------------------------------------------------------ */
static int right_of(int Lx, int Ly, int per_x, uint64_t i, uint64_t *j) {
  uint64_t x = i % (uint64_t)Lx;
  (void)Ly;
  if (x + 1 < (uint64_t)Lx) { *j = i + 1; return 1; }
  if (!per_x) return 0;
  *j = i - x; /* wrap to column 0 of the same row */
  return 1;
}

static int down_of(int Lx, int Ly, int per_y, uint64_t i, uint64_t *j) {
  uint64_t y = i / (uint64_t)Lx;
  if (y + 1 < (uint64_t)Ly) { *j = i + (uint64_t)Lx; return 1; }
  if (!per_y) return 0;
  *j = i % (uint64_t)Lx; /* wrap to row 0 */
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Step 2: bonds.  a = cos(theta) cos(phi) + sin(theta) sin(phi) in FP64 of  */
/* the stored angle; p = 1 - exp(-2 beta a_i a_j) when a_i a_j > 0.          */
/* ------------------------------------------------------------------------ */
static double projection(double theta, double cphi, double sphi) {
  double a = cos(theta) * cphi;
  double b = sin(theta) * sphi;
  return a + b;
}

static double bond_probability(double ai, double aj, double beta) {
  double x = ai * aj;
  if (!(x > 0.0)) return 0.0;
  return 1.0 - exp(-2.0 * beta * x);
}

/* The BOND-domain words of site i = y*Lx + x.  One Philox draw serves the
 * vertical pair of sites (x, 2m) and (x, 2m + 1): counter word 0 is
 * m*Lx + x.  Row 2m takes words 0 and 1 of the draw, row 2m + 1 words 2 and
 * 3; the first is the site's right-bond word, the second its down-bond
 * word.  A bond's uniform comes from bits 31..1 of its word, and bit 0 of
 * the right-bond word is the site's cluster coin (independent of both
 * uniforms). */
static void bond_words(uint64_t seed, uint32_t t, int Lx, uint64_t i,
                       uint32_t *w_right, uint32_t *w_down) {
  uint64_t x = i % (uint64_t)Lx, y = i / (uint64_t)Lx;
  uint64_t c = (y >> 1) * (uint64_t)Lx + x;
  uint32_t w[4];
  philox_draw(seed, (uint32_t)c, (uint32_t)(c >> 32), t, ORC_DOM_BOND, w);
  *w_right = (y & 1u) ? w[2] : w[0];
  *w_down = (y & 1u) ? w[3] : w[1];
}

static double uniform_open(uint32_t w) {
  return ((double)(w >> 1) + 0.5) * 0x1.0p-31; /* in (0, 1), exact */
}

/* Generic bonds over angles already widened to FP64 (ang[i]), for the
 * axis (cphi, sphi) of sweep t. */
static long bonds_generic(int Lx, int Ly, int per_x, int per_y,
                          const double *ang, double cphi, double sphi,
                          double beta, uint64_t seed, uint32_t t,
                          uint8_t *right, uint8_t *down) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  long band = 0;
#pragma omp parallel for schedule(static) reduction(+ : band)
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t w_right, w_down;
    bond_words(seed, t, Lx, i, &w_right, &w_down);
    double ai = projection(ang[i], cphi, sphi);
    uint64_t j;
    right[i] = 0;
    if (right_of(Lx, Ly, per_x, i, &j)) {
      double aj = projection(ang[j], cphi, sphi);
      double p = bond_probability(ai, aj, beta);
      double u = uniform_open(w_right);
      right[i] = (ai * aj > 0.0) && (u < p);
      if (ai * aj > 0.0 && fabs(u - p) < 1e-12) ++band;
    }
    down[i] = 0;
    if (down_of(Lx, Ly, per_y, i, &j)) {
      double aj = projection(ang[j], cphi, sphi);
      double p = bond_probability(ai, aj, beta);
      double u = uniform_open(w_down);
      down[i] = (ai * aj > 0.0) && (u < p);
      if (ai * aj > 0.0 && fabs(u - p) < 1e-12) ++band;
    }
  }
  return band;
}

static double *widen_f32(const float *theta, uint64_t n) {
  double *ang = (double *)malloc(n * sizeof(double));
#pragma omp parallel for schedule(static)
  for (uint64_t i = 0; i < n; ++i) ang[i] = (double)theta[i];
  return ang;
}

static double *widen_f16(const uint16_t *bits, uint64_t n) {
  double *ang = (double *)malloc(n * sizeof(double));
#pragma omp parallel for schedule(static)
  for (uint64_t i = 0; i < n; ++i) ang[i] = (double)half_bits_to_float(bits[i]);
  return ang;
}

static double *widen_u16(const uint16_t *q, uint64_t n) {
  double *ang = (double *)malloc(n * sizeof(double));
#pragma omp parallel for schedule(static)
  for (uint64_t i = 0; i < n; ++i) ang[i] = (double)q[i] * ORC_U16_STEP;
  return ang;
}

long orc_bonds_f32(int Lx, int Ly, int per_x, int per_y, const float *theta,
                   double beta, uint64_t seed, uint32_t t, uint8_t *right,
                   uint8_t *down) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  double ax[4];
  float c32;
  orc_axis(seed, t, ax, &c32);
  double *ang = widen_f32(theta, n);
  long band = bonds_generic(Lx, Ly, per_x, per_y, ang, ax[1], ax[2], beta,
                            seed, t, right, down);
  free(ang);
  return band;
}

long orc_bonds_f16(int Lx, int Ly, int per_x, int per_y,
                   const uint16_t *theta_bits, double beta, uint64_t seed,
                   uint32_t t, uint8_t *right, uint8_t *down) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  double ax[4];
  float c32;
  orc_axis(seed, t, ax, &c32);
  double *ang = widen_f16(theta_bits, n);
  long band = bonds_generic(Lx, Ly, per_x, per_y, ang, ax[1], ax[2], beta,
                            seed, t, right, down);
  free(ang);
  return band;
}

long orc_bonds_u16(int Lx, int Ly, int per_x, int per_y, const uint16_t *q,
                   double beta, uint64_t seed, uint32_t t, uint8_t *right,
                   uint8_t *down) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  double ax[4];
  uint16_t cq;
  orc_axis_u16(seed, t, ax, &cq);
  double *ang = widen_u16(q, n);
  long band = bonds_generic(Lx, Ly, per_x, per_y, ang, ax[1], ax[2], beta,
                            seed, t, right, down);
  free(ang);
  return band;
}

/* u and p of the right (dir 0) or down (dir 1) bond of site i, over angles
 * widened to FP64 by `angle` and the axis (cphi, sphi) of sweep t. */
static void bond_up_generic(int Lx, int Ly, int per_x, int per_y,
                            double (*angle)(const void *, uint64_t),
                            const void *theta, double cphi, double sphi,
                            double beta, uint64_t seed, uint32_t t, int64_t i,
                            int dir, double *u, double *p) {
  uint32_t w_right, w_down;
  bond_words(seed, t, Lx, (uint64_t)i, &w_right, &w_down);
  uint64_t j;
  int ok = dir == 0 ? right_of(Lx, Ly, per_x, (uint64_t)i, &j)
                    : down_of(Lx, Ly, per_y, (uint64_t)i, &j);
  *u = uniform_open(dir == 0 ? w_right : w_down);
  *p = 0.0;
  if (!ok) return;
  double ai = projection(angle(theta, (uint64_t)i), cphi, sphi);
  double aj = projection(angle(theta, j), cphi, sphi);
  *p = bond_probability(ai, aj, beta);
}

static double angle_f32(const void *theta, uint64_t i) {
  return (double)((const float *)theta)[i];
}

static double angle_u16(const void *theta, uint64_t i) {
  return (double)((const uint16_t *)theta)[i] * ORC_U16_STEP;
}

void orc_bond_up_f32(int Lx, int Ly, int per_x, int per_y, const float *theta,
                     double beta, uint64_t seed, uint32_t t, int64_t i,
                     int dir, double *u, double *p) {
  double ax[4];
  float c32;
  orc_axis(seed, t, ax, &c32);
  bond_up_generic(Lx, Ly, per_x, per_y, angle_f32, theta, ax[1], ax[2], beta,
                  seed, t, i, dir, u, p);
}

void orc_bond_up_u16(int Lx, int Ly, int per_x, int per_y, const uint16_t *q,
                     double beta, uint64_t seed, uint32_t t, int64_t i,
                     int dir, double *u, double *p) {
  double ax[4];
  uint16_t cq;
  orc_axis_u16(seed, t, ax, &cq);
  bond_up_generic(Lx, Ly, per_x, per_y, angle_u16, q, ax[1], ax[2], beta,
                  seed, t, i, dir, u, p);
}

/* Bonds of rows y0 .. y0 + nrows - 1 (mod L) of an L x L periodic lattice
 * from the FP32 angles of rows y0 .. y0 + nrows only (theta_rows, row-major,
 * (nrows + 1) x L): the same FP64 rule, random words and axis as the
 * whole-lattice bonds of sweep t, for checks at sizes whose full lattice
 * does not fit in host memory.  right / down: nrows x L bytes; gap_right /
 * gap_down (may be NULL): u - p of each bond.  Returns the number of bonds
 * inside the |u - p| < 1e-12 band. */
long orc_bonds_rows_f32(int L, const float *theta_rows, int64_t y0, int nrows,
                        double beta, uint64_t seed, uint32_t t, uint8_t *right,
                        uint8_t *down, double *gap_right, double *gap_down) {
  double ax[4];
  float c32;
  orc_axis(seed, t, ax, &c32);
  long band = 0;
  for (int r = 0; r < nrows; ++r) {
    uint64_t y = (uint64_t)((y0 + r) % L);
    for (int x = 0; x < L; ++x) {
      uint32_t w_right, w_down;
      bond_words(seed, t, L, y * (uint64_t)L + (uint64_t)x, &w_right, &w_down);
      double ai = projection((double)theta_rows[(uint64_t)r * L + x], ax[1], ax[2]);
      double ar = projection((double)theta_rows[(uint64_t)r * L + (x + 1) % L], ax[1], ax[2]);
      double ad = projection((double)theta_rows[(uint64_t)(r + 1) * L + x], ax[1], ax[2]);
      double pr = bond_probability(ai, ar, beta), pd = bond_probability(ai, ad, beta);
      double ur = uniform_open(w_right), ud = uniform_open(w_down);
      right[(uint64_t)r * L + x] = (ai * ar > 0.0) && (ur < pr);
      down[(uint64_t)r * L + x] = (ai * ad > 0.0) && (ud < pd);
      if (gap_right) gap_right[(uint64_t)r * L + x] = ur - pr;
      if (gap_down) gap_down[(uint64_t)r * L + x] = ud - pd;
      if (ai * ar > 0.0 && fabs(ur - pr) < 1e-12) ++band;
      if (ai * ad > 0.0 && fabs(ud - pd) < 1e-12) ++band;
    }
  }
  return band;
}

/* ------------------------------------------------------------------------ */
/* Step 3: connected components.  Label = minimum site index.                */
/* ------------------------------------------------------------------------ */
long orc_label_bfs(int Lx, int Ly, int per_x, int per_y, const uint8_t *right,
                   const uint8_t *down, uint32_t *label, uint32_t *queue) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  uint8_t *seen = (uint8_t *)calloc(n, 1);
  long comps = 0;
  for (uint64_t s = 0; s < n; ++s) {
    if (seen[s]) continue;
    /* s is the smallest unvisited index, hence the minimum of its component */
    ++comps;
    uint64_t head = 0, tail = 0;
    queue[tail++] = (uint32_t)s;
    seen[s] = 1;
    while (head < tail) {
      uint64_t i = queue[head++];
      label[i] = (uint32_t)s;
      uint64_t x = i % (uint64_t)Lx, y = i / (uint64_t)Lx;
      uint64_t nb[4];
      int has[4];
      /* right: bond stored at i */
      has[0] = right_of(Lx, Ly, per_x, i, &nb[0]) && right[i];
      /* down: bond stored at i */
      has[1] = down_of(Lx, Ly, per_y, i, &nb[1]) && down[i];
      /* left: bond stored at the left neighbour */
      has[2] = 0;
      if (x > 0) {
        nb[2] = i - 1;
        has[2] = right[i - 1];
      } else if (per_x) {
        nb[2] = i + (uint64_t)Lx - 1;
        has[2] = right[nb[2]];
      }
      /* up: bond stored at the upper neighbour */
      has[3] = 0;
      if (y > 0) {
        nb[3] = i - (uint64_t)Lx;
        has[3] = down[nb[3]];
      } else if (per_y) {
        nb[3] = i + (uint64_t)Lx * (uint64_t)(Ly - 1);
        has[3] = down[nb[3]];
      }
      for (int k = 0; k < 4; ++k) {
        if (has[k] && !seen[nb[k]]) {
          seen[nb[k]] = 1;
          queue[tail++] = (uint32_t)nb[k];
        }
      }
    }
  }
  free(seen);
  return comps;
}

static uint32_t uf_find(uint32_t *parent, uint32_t i) {
  while (parent[i] != i) {
    parent[i] = parent[parent[i]]; /* path halving */
    i = parent[i];
  }
  return i;
}

static void uf_union(uint32_t *parent, uint32_t a, uint32_t b) {
  uint32_t ra = uf_find(parent, a), rb = uf_find(parent, b);
  if (ra == rb) return;
  if (ra < rb) parent[rb] = ra; /* the smaller index stays the root */
  else parent[ra] = rb;
}

long orc_label_uf(int Lx, int Ly, int per_x, int per_y, const uint8_t *right,
                  const uint8_t *down, uint32_t *label) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  for (uint64_t i = 0; i < n; ++i) label[i] = (uint32_t)i;
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t j;
    if (right[i] && right_of(Lx, Ly, per_x, i, &j))
      uf_union(label, (uint32_t)i, (uint32_t)j);
    if (down[i] && down_of(Lx, Ly, per_y, i, &j))
      uf_union(label, (uint32_t)i, (uint32_t)j);
  }
  long comps = 0;
  for (uint64_t i = 0; i < n; ++i) {
    label[i] = uf_find(label, (uint32_t)i);
    if (label[i] == i) ++comps;
  }
  return comps;
}

/* ------------------------------------------------------------------------ */
/* Step 4: flip.  Reflection about the axis: theta' = C - theta (mod 2 pi).  */
/* ------------------------------------------------------------------------ */
int orc_coin(uint64_t seed, uint32_t t, int Lx, uint32_t root) {
  uint32_t w_right, w_down;
  bond_words(seed, t, Lx, root, &w_right, &w_down);
  return (int)(w_right & 1u);
}

long orc_flip_f32(int Lx, int Ly, float *theta, const uint32_t *label,
                  uint64_t seed, uint32_t t, float c32, uint8_t *flipped) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  long count = 0;
#pragma omp parallel for schedule(static) reduction(+ : count)
  for (uint64_t i = 0; i < n; ++i) {
    int f = orc_coin(seed, t, Lx, label[i]);
    if (flipped) flipped[i] = (uint8_t)f;
    if (f) {
      theta[i] = wrap_f32(c32 - theta[i]);
      ++count;
    }
  }
  return count;
}

long orc_flip_f16(int Lx, int Ly, uint16_t *theta_bits, const uint32_t *label,
                  uint64_t seed, uint32_t t, float c32, uint8_t *flipped) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  long count = 0;
#pragma omp parallel for schedule(static) reduction(+ : count)
  for (uint64_t i = 0; i < n; ++i) {
    int f = orc_coin(seed, t, Lx, label[i]);
    if (flipped) flipped[i] = (uint8_t)f;
    if (f) {
      float v = wrap_f32(c32 - half_bits_to_float(theta_bits[i]));
      theta_bits[i] = store_angle_f16(v);
      ++count;
    }
  }
  return count;
}

/* u16: reflection about the grid axis, q' = (Cq - q) mod 65536, exact. */
long orc_flip_u16(int Lx, int Ly, uint16_t *q, const uint32_t *label,
                  uint64_t seed, uint32_t t, uint16_t cq, uint8_t *flipped) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  long count = 0;
#pragma omp parallel for schedule(static) reduction(+ : count)
  for (uint64_t i = 0; i < n; ++i) {
    int f = orc_coin(seed, t, Lx, label[i]);
    if (flipped) flipped[i] = (uint8_t)f;
    if (f) {
      q[i] = (uint16_t)(((uint32_t)cq + 65536u - (uint32_t)q[i]) & 0xFFFFu);
      ++count;
    }
  }
  return count;
}

/* ------------------------------------------------------------------------ */
/* Step 5: observables (Eqs. (3)-(6)).  Terms in FP64, sums in long double.  */
/* ------------------------------------------------------------------------ */
static void sums_generic(int Lx, int Ly, int per_x, int per_y,
                         const double *ang, orc_sums *s) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  long double c = 0, sn = 0, cr = 0, sr = 0, cd = 0, sd = 0;
  long double ac = 0, asn = 0, acr = 0, asr = 0, acd = 0, asd = 0;
  long double fx[4] = {0, 0, 0, 0}, fy[4] = {0, 0, 0, 0};
  uint64_t nr = 0, nd = 0;
#pragma omp parallel for schedule(static) \
    reduction(+ : c, sn, cr, sr, cd, sd, ac, asn, acr, asr, acd, asd, nr, nd, fx[:4], fy[:4])
  for (uint64_t i = 0; i < n; ++i) {
    double ci = cos(ang[i]), si = sin(ang[i]);
    c += ci;
    sn += si;
    ac += fabs(ci);
    asn += fabs(si);
    uint64_t x = i % (uint64_t)Lx, y = i / (uint64_t)Lx;
    double kx = ORC_TWO_PI * (double)x / (double)Lx;
    double ky = ORC_TWO_PI * (double)y / (double)Ly;
    fx[0] += ci * cos(kx);
    fx[1] += ci * sin(kx);
    fx[2] += si * cos(kx);
    fx[3] += si * sin(kx);
    fy[0] += ci * cos(ky);
    fy[1] += ci * sin(ky);
    fy[2] += si * cos(ky);
    fy[3] += si * sin(ky);
    uint64_t j;
    if (right_of(Lx, Ly, per_x, i, &j)) {
      double d = ang[i] - ang[j];
      cr += cos(d);
      sr += sin(d);
      acr += fabs(cos(d));
      asr += fabs(sin(d));
      ++nr;
    }
    if (down_of(Lx, Ly, per_y, i, &j)) {
      double d = ang[i] - ang[j];
      cd += cos(d);
      sd += sin(d);
      acd += fabs(cos(d));
      asd += fabs(sin(d));
      ++nd;
    }
  }
  s->sum_cos = (double)c;
  s->sum_sin = (double)sn;
  s->sum_cos_r = (double)cr;
  s->sum_sin_r = (double)sr;
  s->sum_cos_d = (double)cd;
  s->sum_sin_d = (double)sd;
  s->n_sites = (double)n;
  s->n_links_r = (double)nr;
  s->n_links_d = (double)nd;
  s->abs_cos = (double)ac;
  s->abs_sin = (double)asn;
  s->abs_cos_r = (double)acr;
  s->abs_sin_r = (double)asr;
  s->abs_cos_d = (double)acd;
  s->abs_sin_d = (double)asd;
  for (int k = 0; k < 4; ++k) {
    s->fx[k] = (double)fx[k];
    s->fy[k] = (double)fy[k];
  }
}

void orc_sums_f32(int Lx, int Ly, int per_x, int per_y, const float *theta,
                  orc_sums *s) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  double *ang = widen_f32(theta, n);
  sums_generic(Lx, Ly, per_x, per_y, ang, s);
  free(ang);
}

void orc_sums_f16(int Lx, int Ly, int per_x, int per_y,
                  const uint16_t *theta_bits, orc_sums *s) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  double *ang = widen_f16(theta_bits, n);
  sums_generic(Lx, Ly, per_x, per_y, ang, s);
  free(ang);
}

void orc_sums_u16(int Lx, int Ly, int per_x, int per_y, const uint16_t *q,
                  orc_sums *s) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  double *ang = widen_u16(q, n);
  sums_generic(Lx, Ly, per_x, per_y, ang, s);
  free(ang);
}

void orc_derive(const orc_sums *s, double beta, orc_obs *o) {
  double n = s->n_sites;
  o->energy_per_site = -(s->sum_cos_r + s->sum_cos_d) / n;
  o->mx = s->sum_cos / n;
  o->my = s->sum_sin / n;
  o->m2 = o->mx * o->mx + o->my * o->my;
  o->ex = s->sum_cos_r / n;
  o->sx = s->sum_sin_r / n;
  o->ey = s->sum_cos_d / n;
  o->sy = s->sum_sin_d / n;
  /* Eq. (4) with J = 1, T = 1/beta and L^2 = N: Upsilon = e - beta N s^2 */
  o->upsilon = o->ex - beta * n * o->sx * o->sx;
  o->beta = beta;
  double ax = 0.0, ay = 0.0;
  for (int k = 0; k < 4; ++k) {
    ax += s->fx[k] * s->fx[k];
    ay += s->fy[k] * s->fy[k];
  }
  o->chik = (ax + ay) / (2.0 * n);
  o->flipped = 0.0; /* set by the update that produced the configuration */
  o->l1_mx = s->abs_cos / n;
  o->l1_my = s->abs_sin / n;
  o->l1_ex = s->abs_cos_r / n;
  o->l1_sx = s->abs_sin_r / n;
  o->l1_ey = s->abs_cos_d / n;
  o->l1_sy = s->abs_sin_d / n;
}

/* ------------------------------------------------------------------------ */
/* Step 6: PCC.                                                              */
/* ------------------------------------------------------------------------ */
double orc_pcc_next_beta(double beta, double beta_upsilon, double target,
                         double dbeta) {
  /* smaller than the target: increase beta; otherwise (ties too) decrease */
  if (beta_upsilon < target) return beta + dbeta;
  return beta - dbeta;
}

double orc_pcc_dbeta(double dbeta0, uint32_t halve_every, uint32_t k) {
  if (halve_every == 0) return dbeta0;
  return ldexp(dbeta0, -(int)(k / halve_every));
}

/* ------------------------------------------------------------------------ */
/* Threads.  The same source is built twice: plainly (the oracle the tests   */
/* use; the OpenMP pragmas above are ignored) and with -fopenmp, where the   */
/* bond, flip and observable loops run on all host cores and the labeling    */
/* stays sequential.  The OpenMP build only times the CPU baseline; its      */
/* parallel sums add the same terms in another order.                        */
/* ------------------------------------------------------------------------ */
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Whole sweeps.                                                             */
/* ------------------------------------------------------------------------ */
void orc_sw_run_f32(int Lx, int Ly, int per_x, int per_y, float *theta,
                    double beta, uint64_t seed, uint32_t t0, uint32_t n,
                    uint8_t *right, uint8_t *down, uint32_t *label,
                    uint32_t *queue, orc_obs *obs) {
  for (uint32_t s = 0; s < n; ++s) {
    uint32_t t = t0 + s;
    double ax[4];
    float c32;
    orc_axis(seed, t, ax, &c32);
    orc_bonds_f32(Lx, Ly, per_x, per_y, theta, beta, seed, t, right, down);
    orc_label_bfs(Lx, Ly, per_x, per_y, right, down, label, queue);
    long flipped = orc_flip_f32(Lx, Ly, theta, label, seed, t, c32, NULL);
    if (obs) {
      orc_sums sm;
      orc_sums_f32(Lx, Ly, per_x, per_y, theta, &sm);
      orc_derive(&sm, beta, &obs[s]);
      obs[s].flipped = (double)flipped;
    }
  }
}

void orc_sw_run_f16(int Lx, int Ly, int per_x, int per_y,
                    uint16_t *theta_bits, double beta, uint64_t seed,
                    uint32_t t0, uint32_t n, uint8_t *right, uint8_t *down,
                    uint32_t *label, uint32_t *queue, orc_obs *obs) {
  for (uint32_t s = 0; s < n; ++s) {
    uint32_t t = t0 + s;
    double ax[4];
    float c32;
    orc_axis(seed, t, ax, &c32);
    orc_bonds_f16(Lx, Ly, per_x, per_y, theta_bits, beta, seed, t, right,
                  down);
    orc_label_bfs(Lx, Ly, per_x, per_y, right, down, label, queue);
    long flipped = orc_flip_f16(Lx, Ly, theta_bits, label, seed, t, c32, NULL);
    if (obs) {
      orc_sums sm;
      orc_sums_f16(Lx, Ly, per_x, per_y, theta_bits, &sm);
      orc_derive(&sm, beta, &obs[s]);
      obs[s].flipped = (double)flipped;
    }
  }
}

void orc_sw_run_u16(int Lx, int Ly, int per_x, int per_y, uint16_t *q,
                    double beta, uint64_t seed, uint32_t t0, uint32_t n,
                    uint8_t *right, uint8_t *down, uint32_t *label,
                    uint32_t *queue, orc_obs *obs) {
  for (uint32_t s = 0; s < n; ++s) {
    uint32_t t = t0 + s;
    double ax[4];
    uint16_t cq;
    orc_axis_u16(seed, t, ax, &cq);
    orc_bonds_u16(Lx, Ly, per_x, per_y, q, beta, seed, t, right, down);
    orc_label_bfs(Lx, Ly, per_x, per_y, right, down, label, queue);
    long flipped = orc_flip_u16(Lx, Ly, q, label, seed, t, cq, NULL);
    if (obs) {
      orc_sums sm;
      orc_sums_u16(Lx, Ly, per_x, per_y, q, &sm);
      orc_derive(&sm, beta, &obs[s]);
      obs[s].flipped = (double)flipped;
    }
  }
}

void orc_pcc_run_f32(int L, float *theta, double *beta, double target,
                     double dbeta0, uint32_t halve_every, uint32_t block,
                     uint64_t seed, uint32_t t0, uint32_t k0, uint32_t n,
                     double *blk_acc, uint32_t *blk_count, uint8_t *right,
                     uint8_t *down, uint32_t *label, uint32_t *queue,
                     orc_obs *obs) {
  for (uint32_t s = 0; s < n; ++s) {
    orc_obs o;
    orc_sw_run_f32(L, L, 1, 1, theta, *beta, seed, t0 + s, 1, right, down,
                   label, queue, &o);
    if (obs) obs[s] = o;
    *blk_acc += o.beta * o.upsilon;
    *blk_count += 1;
    if (*blk_count >= block) {
      double mean = *blk_acc / (double)block;
      double db = orc_pcc_dbeta(dbeta0, halve_every, k0 + s);
      *beta = orc_pcc_next_beta(*beta, mean, target, db);
      *blk_acc = 0.0;
      *blk_count = 0;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Wolff single-cluster update (Sec. 2 names Wolff's single-cluster          */
/* algorithm beside SW).  Update t uses the axis and the bond random numbers */
/* of SW sweep t; its seed site comes from word 2 of the AXIS draw.  The     */
/* cluster is grown the way the single-cluster algorithm grows it: a         */
/* breadth-first search from the seed that tests each bond on the cluster's  */
/* boundary as it meets it, with the same FP64 rule and the same random word */
/* that the SW bonds use.  The cluster is always reflected.                  */
/* ------------------------------------------------------------------------ */
uint64_t orc_seed_site(uint64_t seed, uint32_t t, uint64_t n) {
  uint32_t w[4];
  philox_draw(seed, 0u, 0u, t, ORC_DOM_AXIS, w);
  return ((uint64_t)w[2] * n) >> 32; /* uniform over 0 .. n-1 (n <= 2^32) */
}

static int left_of(int Lx, int per_x, uint64_t i, uint64_t *j) {
  uint64_t x = i % (uint64_t)Lx;
  if (x > 0) { *j = i - 1; return 1; }
  if (!per_x) return 0;
  *j = i + (uint64_t)Lx - 1;
  return 1;
}

static int up_of(int Lx, int Ly, int per_y, uint64_t i, uint64_t *j) {
  uint64_t y = i / (uint64_t)Lx;
  if (y > 0) { *j = i - (uint64_t)Lx; return 1; }
  if (!per_y) return 0;
  *j = i + (uint64_t)Lx * (uint64_t)(Ly - 1);
  return 1;
}

/* Is the right (dir 0) or down (dir 1) bond of site `owner` active?  The
 * same test as bonds_generic, for one bond. */
static int bond_active(int Lx, int Ly, int per_x, int per_y, const double *ang,
                       double cphi, double sphi, double beta, uint64_t seed,
                       uint32_t t, uint64_t owner, int dir) {
  uint64_t j;
  int ok = dir == 0 ? right_of(Lx, Ly, per_x, owner, &j)
                    : down_of(Lx, Ly, per_y, owner, &j);
  if (!ok) return 0;
  uint32_t w_right, w_down;
  bond_words(seed, t, Lx, owner, &w_right, &w_down);
  double ai = projection(ang[owner], cphi, sphi);
  double aj = projection(ang[j], cphi, sphi);
  double p = bond_probability(ai, aj, beta);
  double u = uniform_open(dir == 0 ? w_right : w_down);
  return (ai * aj > 0.0) && (u < p);
}

long orc_wolff_cluster(int Lx, int Ly, int per_x, int per_y, const double *ang,
                       double cphi, double sphi, double beta, uint64_t seed,
                       uint32_t t, uint64_t i0, uint8_t *in_cluster,
                       uint32_t *queue) {
  uint64_t n = (uint64_t)Lx * (uint64_t)Ly;
  memset(in_cluster, 0, n);
  uint64_t head = 0, tail = 0;
  in_cluster[i0] = 1;
  queue[tail++] = (uint32_t)i0;
  while (head < tail) {
    uint64_t i = queue[head++];
    for (int k = 0; k < 4; ++k) {
      /* the bond to each neighbour, named by its owner (the left or upper
       * site) and direction */
      uint64_t owner = i, other;
      int dir = k & 1;
      int ok;
      if (k == 0) ok = right_of(Lx, Ly, per_x, i, &other);
      else if (k == 1) ok = down_of(Lx, Ly, per_y, i, &other);
      else if (k == 2) { ok = left_of(Lx, per_x, i, &other); owner = other; }
      else { ok = up_of(Lx, Ly, per_y, i, &other); owner = other; }
      if (!ok || in_cluster[other]) continue;
      if (bond_active(Lx, Ly, per_x, per_y, ang, cphi, sphi, beta, seed, t,
                      owner, dir)) {
        in_cluster[other] = 1;
        queue[tail++] = (uint32_t)other;
      }
    }
  }
  return (long)tail;
}

/* n Wolff updates t0 .. t0+n-1 of angles in storage format dtype (0 FP32,
 * 1 FP16 bits, 2 u16), recording the configuration after each. */
static void wolff_run(int dtype, int Lx, int Ly, int per_x, int per_y,
                      void *theta, double beta, uint64_t seed, uint32_t t0,
                      uint32_t n, uint8_t *in_cluster, uint32_t *queue,
                      orc_obs *obs) {
  uint64_t N = (uint64_t)Lx * (uint64_t)Ly;
  for (uint32_t s = 0; s < n; ++s) {
    uint32_t t = t0 + s;
    double ax[4];
    float c32 = 0.0f;
    uint16_t cq = 0;
    double *ang;
    if (dtype == 2) {
      orc_axis_u16(seed, t, ax, &cq);
      ang = widen_u16((const uint16_t *)theta, N);
    } else {
      orc_axis(seed, t, ax, &c32);
      ang = dtype == 0 ? widen_f32((const float *)theta, N)
                       : widen_f16((const uint16_t *)theta, N);
    }
    uint64_t i0 = orc_seed_site(seed, t, N);
    long size = orc_wolff_cluster(Lx, Ly, per_x, per_y, ang, ax[1], ax[2],
                                  beta, seed, t, i0, in_cluster, queue);
    free(ang);
    for (uint64_t i = 0; i < N; ++i) {
      if (!in_cluster[i]) continue;
      if (dtype == 0) {
        float *th = (float *)theta;
        th[i] = wrap_f32(c32 - th[i]);
      } else if (dtype == 1) {
        uint16_t *hb = (uint16_t *)theta;
        hb[i] = store_angle_f16(wrap_f32(c32 - half_bits_to_float(hb[i])));
      } else {
        uint16_t *q = (uint16_t *)theta;
        q[i] = (uint16_t)(((uint32_t)cq + 65536u - (uint32_t)q[i]) & 0xFFFFu);
      }
    }
    if (obs) {
      orc_sums sm;
      if (dtype == 0) orc_sums_f32(Lx, Ly, per_x, per_y, (const float *)theta, &sm);
      else if (dtype == 1) orc_sums_f16(Lx, Ly, per_x, per_y, (const uint16_t *)theta, &sm);
      else orc_sums_u16(Lx, Ly, per_x, per_y, (const uint16_t *)theta, &sm);
      orc_derive(&sm, beta, &obs[s]);
      obs[s].flipped = (double)size;
    }
  }
}

void orc_wolff_run_f32(int Lx, int Ly, int per_x, int per_y, float *theta,
                       double beta, uint64_t seed, uint32_t t0, uint32_t n,
                       uint8_t *in_cluster, uint32_t *queue, orc_obs *obs) {
  wolff_run(0, Lx, Ly, per_x, per_y, theta, beta, seed, t0, n, in_cluster,
            queue, obs);
}

void orc_wolff_run_f16(int Lx, int Ly, int per_x, int per_y,
                       uint16_t *theta_bits, double beta, uint64_t seed,
                       uint32_t t0, uint32_t n, uint8_t *in_cluster,
                       uint32_t *queue, orc_obs *obs) {
  wolff_run(1, Lx, Ly, per_x, per_y, theta_bits, beta, seed, t0, n,
            in_cluster, queue, obs);
}

void orc_wolff_run_u16(int Lx, int Ly, int per_x, int per_y, uint16_t *q,
                       double beta, uint64_t seed, uint32_t t0, uint32_t n,
                       uint8_t *in_cluster, uint32_t *queue, orc_obs *obs) {
  wolff_run(2, Lx, Ly, per_x, per_y, q, beta, seed, t0, n, in_cluster, queue,
            obs);
}

/* ------------------------------------------------------------------------ */
/* Metropolis single-spin flips (an independent sampler for cross-checks).   */
/* ------------------------------------------------------------------------ */
static double u53(uint32_t hi, uint32_t lo) {
  uint64_t bits = ((uint64_t)hi << 32) | (uint64_t)lo;
  return (double)(bits >> 11) * 0x1.0p-53;
}

void orc_metropolis_run(int Lx, int Ly, double *theta, double beta,
                        double delta, uint64_t seed, uint32_t t0, uint32_t n,
                        orc_obs *obs, long *accepted) {
  uint64_t N = (uint64_t)Lx * (uint64_t)Ly;
  long acc = 0;
  for (uint32_t s = 0; s < n; ++s) {
    uint32_t t = t0 + s;
    for (uint64_t i = 0; i < N; ++i) {
      uint32_t w[4];
      philox_draw(seed, (uint32_t)i, (uint32_t)(i >> 32), t, ORC_DOM_METRO, w);
      double prop = theta[i] + delta * (2.0 * u53(w[0], w[1]) - 1.0);
      prop = fmod(prop, ORC_TWO_PI);
      if (prop < 0.0) prop += ORC_TWO_PI;
      uint64_t x = i % (uint64_t)Lx, y = i / (uint64_t)Lx;
      uint64_t nb[4];
      nb[0] = y * (uint64_t)Lx + (x + 1) % (uint64_t)Lx;
      nb[1] = y * (uint64_t)Lx + (x + (uint64_t)Lx - 1) % (uint64_t)Lx;
      nb[2] = ((y + 1) % (uint64_t)Ly) * (uint64_t)Lx + x;
      nb[3] = ((y + (uint64_t)Ly - 1) % (uint64_t)Ly) * (uint64_t)Lx + x;
      double dE = 0.0;
      for (int k = 0; k < 4; ++k)
        dE -= cos(prop - theta[nb[k]]) - cos(theta[i] - theta[nb[k]]);
      if (dE <= 0.0 || u53(w[2], w[3]) < exp(-beta * dE)) {
        theta[i] = prop;
        ++acc;
      }
    }
    if (obs) {
      orc_sums sm;
      sums_generic(Lx, Ly, 1, 1, theta, &sm);
      orc_derive(&sm, beta, &obs[s]);
    }
  }
  if (accepted) *accepted = acc;
}
