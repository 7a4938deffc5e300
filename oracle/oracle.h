/*
 * oracle.h -- plain, sequential CPU oracle for the Swendsen-Wang sweep of the
 * two-dimensional classical XY model with Wolff's embedded-Ising reflection.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path, never
 * to stand in for it: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg and reference arm (which time it on the host cores) may
 * load it.  It shares no code, header, table or constant
 * generator with the CUDA library; both sides implement Philox4x32-10
 * independently from its published definition (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11).
 *
 * Model (the paper's Eq. (3)): H = -J sum_<ij> cos(theta_i - theta_j), J = 1,
 * nearest neighbours of an Lx x Ly square lattice, site index i = y*Lx + x.
 * Each direction can be periodic or open (open is used only for the 1D chain
 * checks: Ly = 1, open x).
 *
 * One sweep t (one MCS) is, in order:
 *   1. axis:  phi from Philox domain AXIS, r = (cos phi, sin phi),
 *             C = (pi + 2 phi) mod 2 pi, C32 = (float)C.
 *   2. bonds: a_i = s_i . r in FP64; right/down bond <ij> is active iff
 *             a_i a_j > 0 and u < 1 - exp(-2 beta a_i a_j).  One Philox
 *             draw of domain BOND serves the vertical pair of sites (x, 2m),
 *             (x, 2m + 1) (counter word 0 = m Lx + x): row 2m takes words 0
 *             (right) and 1 (down), row 2m + 1 words 2 and 3; a bond's u is
 *             ((w >> 1) + 1/2) 2^-31 of its word w.
 *   3. labels: connected components of the active bonds; label = the minimum
 *             site index of the component (BFS; union-find as a second copy).
 *   4. flip:  a cluster flips iff bit 0 of its root's right-bond word is 1;
 *             a flipped angle becomes wrap(C32 - theta) in FP32, which is the
 *             reflection s' = s - 2 (s.r) r of Wolff's embedding.
 *   5. observables on the flipped configuration: energy, magnetisation and
 *             the helicity-modulus sums of the paper's Eqs. (4)-(6).
 *   6. (PCC) beta <- beta + dbeta if beta*Upsilon < target else beta - dbeta
 *             (the paper's helicity-modulus PCC rule, Sec. 2, after Eq. (6)).
 *
 * All floating point is FP64 except where the stored-angle format fixes FP32
 * (or FP16) arithmetic: the flip and the initial angles.  The u16 variant
 * (theta = q 2pi / 65536, a storage format that is not the paper's) puts the
 * axis on the angle grid so that its flip is exact integer arithmetic.  Built with
 * -ffp-contract=off and without -ffast-math.
 */
#ifndef XY_ORACLE_H
#define XY_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox counter domains (counter word 3). */
enum { ORC_DOM_BOND = 0, ORC_DOM_AXIS = 1, ORC_DOM_INIT = 2,
       ORC_DOM_WORKLOAD = 3, ORC_DOM_METRO = 4 };

/* Observable sums of one configuration (raw, not normalised). */
typedef struct {
  double sum_cos;      /* sum_i cos(theta_i)                    */
  double sum_sin;      /* sum_i sin(theta_i)                    */
  double sum_cos_r;    /* sum over right links cos(th_i - th_R) */
  double sum_sin_r;    /* sum over right links sin(th_i - th_R) */
  double sum_cos_d;    /* sum over down links  cos(th_i - th_D) */
  double sum_sin_d;    /* sum over down links  sin(th_i - th_D) */
  double n_sites;      /* N = Lx*Ly                             */
  double n_links_r;    /* number of right links (N if periodic) */
  double n_links_d;    /* number of down links                  */
  /* Fourier components of the spin field at the smallest wave vectors,
   * k = (2 pi / Lx, 0) and (0, 2 pi / Ly) (the paper's Eq. (9)):
   * fx[0..3] = sum_r (cos th cos kx, cos th sin kx, sin th cos kx,
   * sin th sin kx) with kx = 2 pi x / Lx; fy[] the same with y. */
  double fx[4];
  double fy[4];
  /* L1 norms of the six sums above (sum of |term|): the scale against which
   * a sum that cancels (m, s_x, s_y, or e near infinite temperature) is
   * compared (tolerance reading A19) */
  double abs_cos, abs_sin, abs_cos_r, abs_sin_r, abs_cos_d, abs_sin_d;
} orc_sums;

/* Derived per-configuration observables. */
typedef struct {
  double energy_per_site;  /* -(sum_cos_r + sum_cos_d) / N                 */
  double m2;               /* mx^2 + my^2                                  */
  double mx, my;           /* N^-1 sum cos, N^-1 sum sin                   */
  double ex, sx;           /* N^-1 sum_x cos, N^-1 sum_x sin (Eqs. 5-6)    */
  double ey, sy;           /* same along y                                 */
  double upsilon;          /* ex - beta N sx^2 (Eq. 4, J = 1, T = 1/beta)  */
  double beta;             /* the beta the configuration was sampled at    */
  double chik;             /* (|F(kx)|^2 + |F(ky)|^2) / (2N): the
                              configuration's chi at the smallest nonzero
                              wave vector, averaged over x and y (Eq. (9)) */
  double flipped;          /* sites the update reflected (0 from derive)   */
  /* the L1 norms per site of the sums behind mx, my, ex, sx, ey, sy */
  double l1_mx, l1_my, l1_ex, l1_sx, l1_ey, l1_sy;
} orc_obs;

/* Threads of the loops that run in parallel in the OpenMP build (bonds,
 * flip, observables; the labeling is sequential): n > 0 sets the count;
 * returns the count in use (always 1 in the plain build). */
int orc_threads(int n);

/* ---- Philox4x32-10 ------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);
/* out[4*k + j] = word j of Philox(ctr + k e_word, key(seed)): counter word
 * `word` (0..3) of ctr advances by k, the other words stay fixed. */
void orc_philox_stream(uint64_t seed, const uint32_t ctr[4], int word,
                       uint64_t n_calls, uint32_t *out);

/* ---- one sweep, step by step -------------------------------------------- */
/* Step 1: axis of sweep t.  out: phi, cos phi, sin phi, C (FP64); c32: C32. */
void orc_axis(uint64_t seed, uint32_t t, double out[4], float *c32);
/* u16 fixed-point angles (theta = q 2pi / 65536; a storage variant, not the
 * paper's): the axis on the reflection grid.  out: phi_q = pi m / 65536,
 * cos, sin (FP64), C = Cq 2pi / 65536; cq = (m + 32768) mod 65536, with m the
 * 16 axis-word bits below the top one (phi mod pi floored to the grid). */
void orc_axis_u16(uint64_t seed, uint32_t t, double out[4], uint16_t *cq);

/* Initial angles: start 0 = random (domain INIT), 1 = ordered (theta = 0). */
void orc_init_angles_f32(int Lx, int Ly, uint64_t seed, int start,
                         float *theta);
void orc_init_angles_f16(int Lx, int Ly, uint64_t seed, int start,
                         uint16_t *theta_bits);
/* u16: q = the top 16 bits of the INIT word the FP32 start uses. */
void orc_init_angles_u16(int Lx, int Ly, uint64_t seed, int start,
                         uint16_t *q);

/* Step 2: bonds.  right[i], down[i] in {0,1}.  Returns the number of bonds
 * whose |u - p| < 1e-12 (the reported exception band of exact mode). */
long orc_bonds_f32(int Lx, int Ly, int per_x, int per_y, const float *theta,
                   double beta, uint64_t seed, uint32_t t, uint8_t *right,
                   uint8_t *down);
long orc_bonds_f16(int Lx, int Ly, int per_x, int per_y,
                   const uint16_t *theta_bits, double beta, uint64_t seed,
                   uint32_t t, uint8_t *right, uint8_t *down);
/* u16: angles q 2pi / 65536 in FP64, axis of orc_axis_u16. */
long orc_bonds_u16(int Lx, int Ly, int per_x, int per_y, const uint16_t *q,
                   double beta, uint64_t seed, uint32_t t, uint8_t *right,
                   uint8_t *down);
/* Bond probability bookkeeping for a single bond (for the band report):
 * writes u and p of the right (dir 0) or down (dir 1) bond of site i. */
void orc_bond_up_f32(int Lx, int Ly, int per_x, int per_y, const float *theta,
                     double beta, uint64_t seed, uint32_t t, int64_t i,
                     int dir, double *u, double *p);
void orc_bond_up_u16(int Lx, int Ly, int per_x, int per_y, const uint16_t *q,
                     double beta, uint64_t seed, uint32_t t, int64_t i,
                     int dir, double *u, double *p);

/* Step 3: labels (minimum site index of each component). Returns the number
 * of components. */
long orc_label_bfs(int Lx, int Ly, int per_x, int per_y, const uint8_t *right,
                   const uint8_t *down, uint32_t *label, uint32_t *queue);
long orc_label_uf(int Lx, int Ly, int per_x, int per_y, const uint8_t *right,
                  const uint8_t *down, uint32_t *label);

/* Bonds of rows y0 .. y0 + nrows - 1 (mod L) of an L x L periodic lattice,
 * from the FP32 angles of rows y0 .. y0 + nrows ((nrows + 1) x L floats):
 * identical to the whole-lattice bonds of those rows, for lattices whose
 * full angle array is too large to widen on the host.  gap_right / gap_down
 * (may be NULL) receive u - p of each bond.  Returns the number of bonds
 * inside the |u - p| < 1e-12 band. */
long orc_bonds_rows_f32(int L, const float *theta_rows, int64_t y0, int nrows,
                        double beta, uint64_t seed, uint32_t t, uint8_t *right,
                        uint8_t *down, double *gap_right, double *gap_down);

/* Step 4: flip.  flipped[i] (optional, may be NULL) records the flip set.
 * Returns the number of flipped sites. */
long orc_flip_f32(int Lx, int Ly, float *theta, const uint32_t *label,
                  uint64_t seed, uint32_t t, float c32, uint8_t *flipped);
long orc_flip_f16(int Lx, int Ly, uint16_t *theta_bits, const uint32_t *label,
                  uint64_t seed, uint32_t t, float c32, uint8_t *flipped);
/* u16: q' = (cq - q) mod 65536 for flipped sites (cq from orc_axis_u16). */
long orc_flip_u16(int Lx, int Ly, uint16_t *q, const uint32_t *label,
                  uint64_t seed, uint32_t t, uint16_t cq, uint8_t *flipped);
/* coin of a root site: 1 = the cluster is reflected. */
int orc_coin(uint64_t seed, uint32_t t, int Lx, uint32_t root);

/* Step 5: observables. */
void orc_sums_f32(int Lx, int Ly, int per_x, int per_y, const float *theta,
                  orc_sums *s);
void orc_sums_f16(int Lx, int Ly, int per_x, int per_y,
                  const uint16_t *theta_bits, orc_sums *s);
void orc_sums_u16(int Lx, int Ly, int per_x, int per_y, const uint16_t *q,
                  orc_sums *s);
void orc_derive(const orc_sums *s, double beta, orc_obs *o);

/* Step 6: PCC beta update (the paper's helicity-modulus rule).
 * beta_upsilon: the (block-averaged) beta*Upsilon that drives this step. */
double orc_pcc_next_beta(double beta, double beta_upsilon, double target,
                         double dbeta);
/* dbeta of PCC step k: dbeta0 * 2^-(k / halve_every) (halve_every = 0: fixed). */
double orc_pcc_dbeta(double dbeta0, uint32_t halve_every, uint32_t k);

/* ---- whole sweeps -------------------------------------------------------- */
/* Runs n sweeps t0 .. t0+n-1 at fixed beta (FP32 angles), writing one
 * orc_obs per sweep to obs (may be NULL).  Scratch: right, down (N bytes
 * each), label and queue (N uint32 each). */
void orc_sw_run_f32(int Lx, int Ly, int per_x, int per_y, float *theta,
                    double beta, uint64_t seed, uint32_t t0, uint32_t n,
                    uint8_t *right, uint8_t *down, uint32_t *label,
                    uint32_t *queue, orc_obs *obs);
void orc_sw_run_f16(int Lx, int Ly, int per_x, int per_y,
                    uint16_t *theta_bits, double beta, uint64_t seed,
                    uint32_t t0, uint32_t n, uint8_t *right, uint8_t *down,
                    uint32_t *label, uint32_t *queue, orc_obs *obs);
void orc_sw_run_u16(int Lx, int Ly, int per_x, int per_y, uint16_t *q,
                    double beta, uint64_t seed, uint32_t t0, uint32_t n,
                    uint8_t *right, uint8_t *down, uint32_t *label,
                    uint32_t *queue, orc_obs *obs);

/* PCC run on a periodic L x L lattice: sweeps t0 .. t0+n-1 (Philox sweep
 * counter).  k0 is the number of sweeps already run under PCC; the sweep with
 * PCC index k adds beta_k*Upsilon_k to the block accumulator, and when the
 * block holds `block` sweeps beta steps by the rule above with
 * dbeta = orc_pcc_dbeta(dbeta0, halve_every, k), driven by the block mean.
 * beta, blk_acc and blk_count are updated in place; obs records the beta each
 * sweep ran at. */
void orc_pcc_run_f32(int L, float *theta, double *beta, double target,
                     double dbeta0, uint32_t halve_every, uint32_t block,
                     uint64_t seed, uint32_t t0, uint32_t k0, uint32_t n,
                     double *blk_acc, uint32_t *blk_count, uint8_t *right,
                     uint8_t *down, uint32_t *label, uint32_t *queue,
                     orc_obs *obs);

/* ---- Wolff single-cluster updates (Sec. 2 names the algorithm) -------- */
/* Update t: the axis and bond random numbers of SW sweep t, seed site
 * i0 = (word 2 of the AXIS draw * n) >> 32.  The cluster of i0 is grown by a
 * breadth-first search that tests each boundary bond with the SW bond rule
 * when it meets it, and is always reflected. */
uint64_t orc_seed_site(uint64_t seed, uint32_t t, uint64_t n);
/* in_cluster: N bytes (1 = in the cluster), queue: N uint32.  ang: angles in
 * FP64, (cphi, sphi) the axis.  Returns the cluster size. */
long orc_wolff_cluster(int Lx, int Ly, int per_x, int per_y, const double *ang,
                       double cphi, double sphi, double beta, uint64_t seed,
                       uint32_t t, uint64_t i0, uint8_t *in_cluster,
                       uint32_t *queue);
/* n updates t0 .. t0+n-1 in place; obs (may be NULL) gets one record per
 * update with flipped = the cluster size. */
void orc_wolff_run_f32(int Lx, int Ly, int per_x, int per_y, float *theta,
                       double beta, uint64_t seed, uint32_t t0, uint32_t n,
                       uint8_t *in_cluster, uint32_t *queue, orc_obs *obs);
void orc_wolff_run_f16(int Lx, int Ly, int per_x, int per_y,
                       uint16_t *theta_bits, double beta, uint64_t seed,
                       uint32_t t0, uint32_t n, uint8_t *in_cluster,
                       uint32_t *queue, orc_obs *obs);
void orc_wolff_run_u16(int Lx, int Ly, int per_x, int per_y, uint16_t *q,
                       double beta, uint64_t seed, uint32_t t0, uint32_t n,
                       uint8_t *in_cluster, uint32_t *queue, orc_obs *obs);

/* Metropolis single-spin-flip sweeps (typewriter order, FP64 angles), an
 * independent sampler used only to cross-check the cluster chain. */
void orc_metropolis_run(int Lx, int Ly, double *theta, double beta,
                        double delta, uint64_t seed, uint32_t t0, uint32_t n,
                        orc_obs *obs, long *accepted);

#ifdef __cplusplus
}
#endif
#endif
