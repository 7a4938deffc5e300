/*
 * xy.h -- C ABI of the B300 (sm_103a) Swendsen-Wang sweep for the 2D
 * classical XY model with Wolff's embedded-Ising reflection.
 *
 * The model is the paper's Eq. (3): H = -J sum_<ij> cos(theta_i - theta_j),
 * J = 1, nearest neighbours of an L x L square lattice with periodic
 * boundaries (Komura & Okabe, Sec. 2).  One sweep (one MCS, Sec. 3) is the
 * Swendsen-Wang multi-cluster update (Sec. 1) in Wolff's embedding:
 *   1. draw a random unit vector r = (cos phi, sin phi);
 *   2. activate each nearest-neighbour bond with probability
 *      p = 1 - exp(-2 beta (s_i.r)(s_j.r)) where that product is positive;
 *   3. label the connected clusters (label = minimum site index);
 *   4. reflect each cluster about r (s -> s - 2 (s.r) r) with probability 1/2;
 *   5. accumulate energy, M^2 and the helicity-modulus sums (Eqs. (4)-(6)).
 * The helicity-modulus PCC (Sec. 2, after Eq. (6)) steps beta after each
 * sweep or block of sweeps: up if beta*Upsilon is below the target, down
 * otherwise.
 *
 * Conventions
 *   - Every call returns an xy_status; xy_last_error() gives a message for
 *     the calling thread.  No C++ exception crosses this boundary.
 *   - Ownership: the CALLER owns all device memory (one workspace buffer per
 *     lattice, sized by xy_workspace_size) and the CUDA stream.  The library
 *     owns only the small opaque host handle; xy_destroy frees the handle and
 *     never the caller's buffers.
 *   - All calls are asynchronous on the handle's stream, except the host-copy
 *     getters/setters and xy_measure with sync = 1, which synchronise it.
 *   - Site index i = y * L + x (row-major, x fastest).  Angles live in
 *     [0, 2 pi) radians, stored as FP32 or IEEE FP16.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key = seed
 *     (low word, high word) and counter (site, 0, sweep, domain); every bit of
 *     a sweep is a pure function of (seed, sweep, site), so results do not
 *     depend on launch shapes, batching or reduction order.
 *   - Device-side failures (a bounded wait that ran out) never trap: the
 *     kernel records an error word, finishes its launch and the next
 *     synchronising call returns XY_ETIMEOUT or XY_EINTERNAL.
 */
#ifndef XY_H
#define XY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  XY_OK = 0,
  XY_EINVAL = 1,       /* bad argument; nothing was launched            */
  XY_ENOMEM = 2,       /* workspace or host buffer too small            */
  XY_ECUDA = 3,        /* a CUDA runtime call failed                    */
  XY_ETIMEOUT = 4,     /* a bounded device-side loop hit its limit      */
  XY_EINTERNAL = 5,    /* a device-side consistency check failed        */
  XY_EUNSUPPORTED = 6  /* valid request this build does not implement   */
} xy_status;

typedef struct xy_lattice xy_lattice; /* opaque host handle */

/* Stored angle format.  XY_F32 and XY_F16 hold theta in [0, 2pi) as IEEE
 * floats; a flipped angle is wrap(C32 - theta) in FP32, rounded to the
 * format.  XY_U16 is a fixed-point storage variant that the paper does not
 * have: theta = q 2pi / 65536 with q in 0..65535.  For it, the axis of every
 * sweep is put on the reflection grid: m = bits 47..62 of the 64-bit axis
 * word (phi mod pi floored to pi/65536), phi_q = pi m / 65536 and
 * Cq = (m + 32768) mod 65536.  The flip is then the exact integer map
 * q -> (Cq - q) mod 65536, and the bonds project on phi_q itself.  Each sweep
 * is an exact cluster move of the 65536-state clock model, at two bytes per
 * site and with no rounding in the flip.  The random start takes the top 16
 * bits of the word that the FP32 start scales. */
typedef enum { XY_F32 = 0, XY_F16 = 1, XY_U16 = 2 } xy_angle_t;

/* Bond-threshold arithmetic.  XY_THR_F64 ("exact mode") decides every bond as
 * the FP64 rule u < 1 - exp(-2 beta a_i a_j) does: an FP32 evaluation with a
 * proven error bound settles all bonds outside a narrow band, and the bonds
 * inside it are recomputed in FP64.  XY_THR_F32 uses the FP32 evaluation
 * alone (faster, differs from the FP64 rule on a measured small fraction of
 * bonds). */
typedef enum { XY_THR_F32 = 0, XY_THR_F64 = 1 } xy_thr_t;

/* What one step (xy_sweep, xy_pcc_step, an engine step) does.
 * XY_UPDATE_SW: one Swendsen-Wang sweep with Wolff's embedding.  Every
 *   cluster of the bond configuration is reflected with probability 1/2.
 * XY_UPDATE_WOLFF: one Wolff single-cluster update (Sec. 2 names the
 *   algorithm).  Step t uses the axis and the bond random numbers of SW
 *   sweep t.  Its seed site is i0 = (w2 * N) >> 32, with w2 word 2 of the
 *   step's AXIS draw.  Only the cluster containing i0 is reflected, and it
 *   always is.  That cluster has the same law as the one the single-cluster
 *   algorithm grows from i0 by testing bonds one at a time, because the
 *   bonds are independent.  The GPU finds it with the same bond and label
 *   kernels as a sweep, so a step costs about as much as a sweep and
 *   reflects on average <cluster size> sites instead of N/2.  Records give
 *   the cluster size in `flipped`. */
typedef enum { XY_UPDATE_SW = 0, XY_UPDATE_WOLFF = 1 } xy_update_t;

typedef struct {
  uint32_t L;              /* linear size, 2 .. 65536 (N = L*L <= 2^32)     */
  uint32_t tile_y;         /* labeling tile height: 16, 32, 64 or 128;
                              0 = the library's choice for this L          */
  uint64_t seed;           /* Philox key                                    */
  double beta;             /* inverse temperature J/T, >= 0                 */
  int32_t angle_dtype;     /* xy_angle_t                                    */
  int32_t threshold_mode;  /* xy_thr_t                                      */
  int32_t start;           /* 0: random angles (Philox domain INIT),
                              1: ordered start (all angles 0)               */
  uint32_t record_cap;     /* observable records kept on the device (ring);
                              0 = 4096                                      */
  uint32_t measure_xi;     /* 1: also record chik (second-moment correlation
                              length, Eqs. (8)-(9)); 0: chik = 0           */
  uint32_t update;         /* xy_update_t                                   */
} xy_config;

/* Observables of the configuration after one sweep (FP64).  N = L*L.
 *   energy_per_site = -(sum_x cos + sum_y cos)/N            (Eq. (3) / N)
 *   mx, my = N^-1 sum (cos theta, sin theta); m2 = mx^2 + my^2
 *   ex, sx = N^-1 sum over x-links of cos, sin (theta_i - theta_{i+x})
 *                                                           (Eqs. (5), (6))
 *   ey, sy = the same over y-links
 *   upsilon = ex - beta N sx^2   (Eq. (4) with J = 1, T = 1/beta, L^2 = N);
 *             the paper's PCC compares beta*upsilon with its target
 *   beta   = the inverse temperature the sweep ran at
 *   sweep  = the sweep counter t of that sweep (0-based)
 *   chik   = (|F(k_x)|^2 + |F(k_y)|^2) / (2N), F(k) = sum_r s(r) e^{ik.r} at
 *            k_x = (2 pi/L, 0), k_y = (0, 2 pi/L): the configuration's
 *            chi(k) at the smallest wave vector (Eq. (9), read as the
 *            thermal average of |F|^2).  With chi0 = N m2,
 *            xi_2nd = sqrt(<chi0>/<chik> - 1) / (2 sin(pi/L))   (Eq. (8)).
 *            Recorded only when the config sets measure_xi, else 0.
 *   flipped = Wolff updates: the number of sites reflected (the cluster
 *            size); 0 for SW sweeps (not counted there, to keep the sweep's
 *            observable kernel lean)                                      */
typedef struct {
  double energy_per_site, m2, mx, my, ex, sx, ey, sy, upsilon, beta;
  uint64_t sweep;
  double chik;
  uint64_t flipped;
} xy_obs;

/* Helicity-modulus PCC (Sec. 2): after every `block` sweeps, with
 * m = mean of beta_t*upsilon_t over the block,
 *   beta <- beta + dbeta  if m <  target
 *   beta <- beta - dbeta  otherwise (ties decrease),
 * dbeta = dbeta0 * 2^-floor(k / halve_every) (halve_every = 0: constant),
 * k = the PCC sweep index of the block's last sweep (sweeps run under PCC
 * since xy_init).  The paper's protocol: target 0.636508, dbeta0 0.0005,
 * halve_every 0, block 1000 (Sec. 3). */
typedef struct {
  double target;
  double dbeta0;
  uint32_t halve_every;
  uint32_t block;
} xy_pcc_params;

/* Message of the last failed call on this thread ("" if none). */
const char *xy_last_error(void);

/* Bytes of device workspace a lattice with this config needs.  The layout is
 * private; the caller provides one buffer of at least this size, 256-byte
 * aligned (any cudaMalloc / torch allocation is).  XY_EINVAL on a bad
 * config. */
xy_status xy_workspace_size(const xy_config *cfg, size_t *bytes);

/* Create a lattice in the caller's workspace and enqueue its initialisation
 * on `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * XY_EINVAL: bad config, NULL pointers or misaligned workspace;
 * XY_ENOMEM: `bytes` below xy_workspace_size.  The workspace must stay
 * allocated until xy_destroy. */
xy_status xy_init(const xy_config *cfg, void *d_workspace, size_t bytes,
                  void *cuda_stream, xy_lattice **out);

/* Enqueue n_sweeps sweeps at the current beta.  Each sweep appends one
 * xy_obs record to the device ring.  Asynchronous.  The records and the
 * next sweep's random axis are made inside the next sweep's first kernel,
 * and one closing kernel per call makes the last record (4 launches per
 * sweep plus 2 per call).  Runs of 16 sweeps inside a call replay a CUDA
 * graph recorded on the handle's private stream at the first call (about
 * 1 ms of host time, once); while the caller captures the lattice's stream,
 * or for sweeps that xy_profile times, every kernel is launched directly. */
xy_status xy_sweep(xy_lattice *h, uint32_t n_sweeps);

/* Enqueue n_sweeps PCC sweeps: each sweep is followed by the PCC rule above.
 * beta lives on the device, so no host round trip happens between sweeps
 * (5 launches per sweep: the record and the beta step need a kernel of
 * their own, because the next sweep's bonds depend on them).  Runs of 16
 * sweeps replay a recorded graph as in xy_sweep.
 * XY_EINVAL on NULL params, block = 0, or negative dbeta0. */
xy_status xy_pcc_step(xy_lattice *h, const xy_pcc_params *p,
                      uint32_t n_sweeps);

/* Copy the records of the sweeps enqueued since the previous xy_measure
 * call into `out` (chronological order).  If more than max_records (or
 * more than the ring capacity) are pending, only the newest ones are
 * returned; *n_out receives the number written.  sync = 1 synchronises the
 * stream first and reports any device-side error (XY_ETIMEOUT /
 * XY_EINTERNAL); sync = 0 skips both, so the caller must have synchronised
 * the stream itself. */
xy_status xy_measure(xy_lattice *h, xy_obs *out, uint32_t max_records,
                     uint32_t *n_out, int sync);

/* Current beta and sweep counter (synchronising). */
xy_status xy_get_state(xy_lattice *h, double *beta, uint64_t *sweep);

/* Destroy the handle (never frees the caller's workspace). */
xy_status xy_destroy(xy_lattice *h);

/* ---- host copies (synchronising) --------------------------------------- */
/* Angles: N elements of the lattice dtype (float, IEEE half bits or u16 q),
 * row-major.  Set float/half values must lie in [0, 2 pi); XY_EINVAL
 * otherwise (every u16 value is valid). */
xy_status xy_get_angles(xy_lattice *h, void *host_dst);
xy_status xy_set_angles(xy_lattice *h, const void *host_src);
/* Spin vectors s_i = (cos theta_i, sin theta_i) of the current angles (the
 * O(2) spins of Eq. (1)), N floats each, row-major, evaluated on the device
 * by the same cos/sin routine the observable sums of xy_measure use
 * (absolute error <= 1e-7).  Either output may be NULL.  Synchronising;
 * allocates a device buffer of at most 32 MiB for the call and frees it
 * before returning. */
xy_status xy_get_spins(xy_lattice *h, float *host_cos, float *host_sin);
/* Bonds of the last sweep as N bytes each (1 = active): right[i] is the bond
 * (x, y)-(x+1 mod L, y), down[i] the bond (x, y)-(x, y+1 mod L). */
xy_status xy_get_bonds(xy_lattice *h, uint8_t *host_right,
                       uint8_t *host_down);
/* Cluster labels of the last sweep: N uint32, label = minimum site index of
 * the cluster. */
xy_status xy_get_labels(xy_lattice *h, uint32_t *host_dst);
/* Sampled state of the last sweep, for checks at sizes whose full arrays are
 * too large to copy: for each of the n site indices in host_sites (each
 * < N; XY_EINVAL otherwise) the stored angle (lattice dtype: float, or the
 * 16 bits of an FP16 or u16 angle), the label, and the bonds as
 * bit 0 = right, bit 1 = down.  Any of the three outputs may be NULL.
 * Synchronising; allocates a device buffer of about 17 n bytes for the call
 * and frees it before returning (a diagnostic, not for the sweep loop). */
xy_status xy_get_sites(xy_lattice *h, const uint64_t *host_sites, uint32_t n,
                       void *host_theta, uint32_t *host_label, uint8_t *host_bonds);
/* Label caller-supplied bond bytes (N each, same meaning as xy_get_bonds)
 * with the device labeling kernels; writes N labels.  Does not touch the
 * angles, the sweep counter or the records. */
xy_status xy_label_bonds(xy_lattice *h, const uint8_t *host_right,
                         const uint8_t *host_down, uint32_t *host_labels);
/* Test and diagnostics: the iteration bound of every device-side global
 * find, union and pointer-jumping loop of this lattice (cap = 0 restores the
 * default, 2^22; a loop that reaches the bound stops, records the error and
 * its launch completes, and the next synchronising call returns
 * XY_ETIMEOUT).  No cluster of a valid lattice needs anywhere near the
 * default; a test sets a tiny bound to make the bound run out on purpose.
 * Synchronising. */
xy_status xy_set_loop_bound(xy_lattice *h, uint32_t cap);
/* Test and diagnostics: the link slots a tile may fill in one sweep's merge
 * (cap = 0 or above the default restores the default, TY + 32: one per
 * edge item, which never overflows).  A smaller cap makes a dense
 * configuration overflow on purpose: the merge records the consistency
 * error, the launches complete, and the next synchronising call returns
 * XY_EINTERNAL (the labels of that sweep are not meaningful).
 * Synchronising. */
xy_status xy_set_link_cap(xy_lattice *h, uint32_t cap);
/* The compute capability the library's device code was built for, as
 * major * 10 + minor of the loaded kernel image (103 for sm_103a).  Needs a
 * CUDA device. */
xy_status xy_build_arch(int *binary_version);
/* Diagnostics of exact mode since xy_init: bonds decided in FP64 (inside
 * the FP32 error band) and, among them, those where the FP32 decision would
 * have differed. */
xy_status xy_get_band_stats(xy_lattice *h, uint64_t *n_fp64,
                            uint64_t *n_fp32_wrong);

/* ---- host-buffer run (end to end) -------------------------------------- */
/* One call that does what a caller with host data does: copy N angles in
 * from host memory (skipped when host_angles_in is NULL), run n_sweeps
 * sweeps, copy the n_sweeps observable records out to host_obs (may be NULL)
 * and the final N angles out to host_angles_out (may be NULL), then
 * synchronise.  Pinned host buffers make the copies asynchronous DMA; the
 * input angles are not range-checked here (values outside [0, 2 pi) give
 * meaningless observables but no fault).  Device-side errors are reported as
 * by xy_measure(sync = 1).  Records returned here are not returned again by
 * xy_measure. */
xy_status xy_run_host(xy_lattice *h, const void *host_angles_in,
                      uint32_t n_sweeps, xy_obs *host_obs,
                      void *host_angles_out);
/* xy_run_host without the final synchronisation: the copies and sweeps are
 * enqueued on the lattice's stream and the call returns at once, so a caller
 * can overlap one lattice's copies with another's sweeps (pinned host
 * buffers make the copies asynchronous).  The host buffers must stay valid,
 * and host_obs / host_angles_out unread, until xy_sync returns; device-side
 * errors are reported by xy_sync. */
xy_status xy_run_host_async(xy_lattice *h, const void *host_angles_in,
                            uint32_t n_sweeps, xy_obs *host_obs,
                            void *host_angles_out);
/* Wait for everything enqueued on the lattice's stream; XY_ETIMEOUT if a
 * device loop hit its bound since the last check.  A device error is
 * reported once: the call that reports it also clears it. */
xy_status xy_sync(xy_lattice *h);

/* ---- kernel timing ------------------------------------------------------- */
/* Kernel index of xy_kernel_times: 0 bond+tile label, 1 edge merge,
 * 2 compress, 3 flip+measure, 4 finalize (timed only in sweeps that launch
 * it: every PCC sweep, and the last sweep of each xy_sweep call). */
#define XY_NUM_KERNELS 5
typedef struct {
  double ms[XY_NUM_KERNELS];          /* summed device time (CUDA events)  */
  uint64_t launches[XY_NUM_KERNELS];  /* launches timed                    */
} xy_kernel_times;
/* enable = k >= 1: from now on bracket every kernel of every k-th sweep
 * with CUDA events on the lattice's stream (resets the totals; the events
 * cost the sweep a few us each, so a stride keeps a timed run honest);
 * enable = 0: stop.  XY_EINVAL for enable < 0. */
xy_status xy_profile(xy_lattice *h, int enable);
/* Synchronise and return the totals since profiling was enabled. */
xy_status xy_profile_read(xy_lattice *h, xy_kernel_times *out);

/* ---- engine: many lattices stepped by shared launches -------------------- */
/* Independent replicas or requests (the paper's runs at several L and beta,
 * Secs. 2-3) advance together: one sweep of every active lattice is one
 * launch of each sweep kernel over all their tiles, replayed from a CUDA
 * graph that is re-recorded only when the active set changes.  Each lattice
 * keeps its own workspace (xy_workspace_size bytes, owned by the caller), its
 * own random numbers and its own fixed-point observable sums, so its results
 * are the same whether it runs alone or with others.  Lattices join
 * (xy_engine_admit) and leave (xy_engine_retire) between steps. */
typedef struct xy_engine xy_engine;
/* Device bytes of the engine's own table for up to max_slots lattices. */
xy_status xy_engine_workspace_size(uint32_t max_slots, size_t *bytes);
/* angle_dtype, threshold_mode and tile_y (16/32/64/128) are shared by all
 * lattices of an engine.  Work is enqueued on cuda_stream; the engine also
 * creates one private stream, used only to record its graph. */
xy_status xy_engine_create(uint32_t max_slots, int angle_dtype,
                           int threshold_mode, uint32_t tile_y,
                           void *d_workspace, size_t bytes, void *cuda_stream,
                           xy_engine **out);
/* Add a lattice (L divisible by 32, else XY_EUNSUPPORTED) in its own
 * workspace; pcc = NULL runs fixed beta, otherwise the PCC rule of
 * xy_pcc_params after each sweep.  cfg->tile_y is ignored (the engine's is
 * used).  *slot receives its slot; XY_ENOMEM when all slots are in use. */
xy_status xy_engine_admit(xy_engine *e, const xy_config *cfg,
                          const xy_pcc_params *pcc, void *d_workspace,
                          size_t bytes, uint32_t *slot);
/* Remove a lattice; its workspace may be reused once this returns. */
xy_status xy_engine_retire(xy_engine *e, uint32_t slot);
/* Enqueue n_sweeps sweeps of every active lattice: a recorded graph of 4
 * sweeps while at least 4 remain, a one-sweep graph for the rest (both
 * recorded again after an admit or retire). */
xy_status xy_engine_step(xy_engine *e, uint32_t n_sweeps);
/* As xy_measure (sync = 1) for one lattice of the engine. */
xy_status xy_engine_measure(xy_engine *e, uint32_t slot, xy_obs *out,
                            uint32_t max_records, uint32_t *n_out);
xy_status xy_engine_get_angles(xy_engine *e, uint32_t slot, void *host_dst);
xy_status xy_engine_get_state(xy_engine *e, uint32_t slot, double *beta,
                              uint64_t *sweep);
xy_status xy_engine_destroy(xy_engine *e);

/* ---- labeling without any device allocation ------------------------------ */
/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory and therefore cannot provide the workspace
 * of a lattice handle -- e.g. a plugin that its host application hands only
 * input and output buffers, or a real-time loop that forbids allocation.
 *
 * Labels the bonds d_right / d_down (device arrays of L*L bytes, nonzero =
 * active, same meaning as xy_get_bonds) of an L x L periodic lattice into
 * d_labels (device array of L*L uint32: minimum site index of each cluster),
 * with the same kernels as xy_label_bonds.  Its scratch is a fixed array
 * built into the library (about 1.05 MB on every GPU that loads it, kept
 * until the process exits); it calls no cudaMalloc/cudaFree.
 *   - L is limited to 2..XY_STATIC_MAX_L; larger L returns XY_EINVAL.
 *   - The first call on a device looks up the scratch's device address
 *     (cudaGetSymbolAddress) for that device; make that first call before
 *     any stream capture (during capture a first call returns XY_EINVAL).
 *     Every later call outside stream capture looks it up again, so a
 *     cudaDeviceReset between calls is followed correctly.  Bond bytes are
 *     active when nonzero (xy_label_bonds, by contrast, takes only 0 / 1).
 *   - All calls share the scratch: calls whose work overlaps on the GPU
 *     (other streams, other host threads) race and give wrong labels.
 *   - Work is enqueued on cuda_stream; sync = 1 waits for it and reports a
 *     device-side loop bound as XY_ETIMEOUT (any other device error as
 *     XY_EINTERNAL), sync = 0 returns after enqueueing (errors then go
 *     unreported). */
#define XY_STATIC_MAX_L 1024u
xy_status xy_label_bonds_static(uint32_t L, const uint8_t *d_right,
                                const uint8_t *d_down, uint32_t *d_labels,
                                void *cuda_stream, int sync);

/* ---- checkpoint --------------------------------------------------------- */
/* Serialise the full chain state (angles, seed, sweep counter, beta, PCC
 * accumulators, dtype) into host memory.  Call with blob = NULL to get the
 * size in *bytes.  Resuming from a checkpoint reproduces the uninterrupted
 * run bit for bit (the random numbers are a function of the sweep counter). */
xy_status xy_save(xy_lattice *h, void *host_blob, size_t *bytes);
xy_status xy_load(xy_lattice *h, const void *host_blob, size_t bytes);

#ifdef __cplusplus
}
#endif
#endif /* XY_H */
