/*
 * soliton.h -- C-ABI of the GB300 (sm_103a) soliton relaxation library.
 *
 * The library relaxes topological solitons of 2D field theories by arrested
 * Newton flow (arxiv 2603.24370, Sec. 3): 4th-order finite-difference stencils
 * with a halo of width two (Sec. 3.1, Eq. 1 and Eq. 2), the flow
 * phi'' = -grad E_h integrated by classic RK4 from rest (Sec. 3.2, Eq. 3), and the
 * arrest v <- 0 whenever E_h rises (Sec. 3.2, Eq. 4), with the unit-length
 * projection of magnetisation models in every RK stage (Sec. 3.2) and GPU-resident
 * reductions of the energy and convergence norm (Sec. 3.3). Theories: Abelian
 * Higgs, Baby Skyrme and the s+id superconductor (Table 1), the chiral magnet
 * (Sec. 4.2, Eq. 5) with optional demagnetisation (Eq. 6), and the rotating trapped
 * BEC (Sec. 4.3) in grand-canonical form or at a fixed atom number. Gradient descent
 * is the alternative minimiser (SS_METHOD_GRADIENT).
 *
 * Conventions shared by every call:
 *  - Every call returns SS_OK (0) or a negative SS_ERR_* code; ss_last_error()
 *    returns a message for the calling thread's last failure.
 *  - A grid is nx x ny sites INCLUDING the width-2 halo. The halo keeps the values
 *    it was given (ss_init_ansatz / ss_set_fields) for ever; interior sites
 *    [2, nx-3] x [2, ny-3] are updated. Site (i, j) sits at
 *    x = (i - (nx-1)/2) dx, y = (j - (ny-1)/2) dy.
 *  - Field arrays are component planes [C][ny][nx], x fastest, in the context's
 *    precision (float for SS_FP32 / SS_FP32_PLAIN, double for SS_FP64; with SS_FP32
 *    the value part is exchanged, and fields set by the caller start with a zero
 *    remainder). C = 4 for the Abelian
 *    Higgs model (Re psi, Im psi, A_1, A_2), C = 3 for the chiral magnet
 *    (n_1, n_2, n_3).
 *  - Pointers passed in are borrowed for the duration of the call only; the
 *    library copies what it keeps. "is_device" = 1 means a device pointer of the
 *    current CUDA device, 0 a host pointer (pinned host memory gives the fastest
 *    copies). The library owns every device buffer it allocates and frees them in
 *    ss_destroy.
 *  - All GPU work of a context runs on the stream given to ss_create_grid; with
 *    NULL the context creates its own blocking stream (ordered with the legacy
 *    default stream; CUDA graphs cannot be captured on the legacy stream itself).
 *    Calls return after their GPU work has completed.
 *  - Contexts are independent: different contexts may be driven at the same time
 *    from different host threads (each on its own stream), so that one context's
 *    host copies overlap another's flow. One context must not be used by two
 *    threads at once.
 *  - The library is built for sm_103a only; it has no CPU fallback.
 */
#ifndef SOLITON_H
#define SOLITON_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SS_OK 0
#define SS_ERR_ARG (-1)           /* invalid argument (sizes, spacings, theory, params) */
#define SS_ERR_STATE (-2)         /* call out of order (e.g. step before theory/fields) */
#define SS_ERR_CUDA (-3)          /* a CUDA runtime call failed; see ss_last_error()   */
#define SS_ERR_TIMEOUT (-4)       /* a bounded device-side wait ran out               */
#define SS_ERR_NONFINITE (-5)     /* energy or force became NaN/Inf; the flow stopped  */
#define SS_ERR_NOT_CONVERGED (-6) /* ss_minimise hit max_steps before the tolerance    */
#define SS_ERR_NOMEM (-7)         /* device or host allocation failed                 */

/* ---- precisions ---- */
#define SS_FP32 1       /* compensated FP32: each field component is stored as two   */
                        /* FP32 planes (value + rounding remainder) so that small    */
                        /* flow increments accumulate; stencils and forces in FP32;  */
                        /* the flow's sums in float-float pairs (TwoSum) totalled in */
                        /* FP64; observables in FP64 (compensated)                   */
#define SS_FP64 2       /* all-FP64 reference form                                    */
#define SS_FP32_PLAIN 3 /* one FP32 plane per component: fastest, but field rounding  */
                        /* limits the attainable dx dy max|G| to about 1e-5           */

/* ---- theories ---- */
#define SS_ABELIAN_HIGGS 1 /* Table 1, params {lambda, u}                                */
#define SS_CHIRAL_MAGNET 2 /* Eq. 5, params {J, D, K, h[, dmi_type[, mu_d]]}:             */
                           /* mu_d = mu_0 M_s^2 > 0 adds demagnetisation (Eq. 6): the      */
                           /* potential psi (lap psi = div n on a Dirichlet box holding the*/
                           /* interior, 5-point Laplacian, psi = 0 just outside the box;   */
                           /* the box is the interior widened by at most a few sites to an */
                           /* FFT-friendly size, and psi is kept on the interior only) is  */
                           /* solved by a sine transform once per step and adds            */
                           /* -mu_d/2 psi div n to the energy, mu_d grad psi to the force  */
                           /* (single-grid contexts only);                                 */
                           /* dmi_type 0 interfacial (d_i = e_3 x e_i), 1 bulk (d_i = e_i),*/
                           /* 2 D_2d "Heusler" (d_1 = e_1, d_2 = -e_2)                     */
#define SS_BABY_SKYRME 3   /* Table 1, params {kappa, mu[, nu]}: unit 3-vector m with       */
                           /* e = |d m|^2/2 + kappa^2/2 |d_1 m x d_2 m|^2 + V(m),            */
                           /* V = mu^2 (1 - m_3) + nu^2/2 m_1^2 (standard potential at nu = 0,*/
                           /* easy-plane at mu = 0); projected like the chiral magnet       */
#define SS_BEC 4           /* rotating trapped BEC (Table 1), params {g, Omega, mu[, N]},   */
                           /* g > 0: psi = u + i v, dimensionless (hbar = m = omega = 1),  */
                           /* e = |grad psi|^2/2 + r^2/2 |psi|^2 + g/2 |psi|^4 - mu |psi|^2 */
                           /*     - Omega Re(psi* L_z psi), L_z = -i (x d_y - y d_x),       */
                           /* (x, y) measured from the grid centre. N = 0 (or absent):      */
                           /* grand-canonical form at chemical potential mu. N > 0: the    */
                           /* atom number dx dy sum_I |psi|^2 is held at N (mu is ignored): */
                           /* every new field is scaled to N on I, its velocity made       */
                           /* tangent to the constraint, and its step takes the force at   */
                           /* the constraint's multiplier mu = sum G_0.psi / (2 sum |psi|^2)*/
                           /* (G_0: mu = 0), held through the step; E_h, the arrest test   */
                           /* and ss_obs.energy are then at mu = 0, and grad_max is the    */
                           /* constrained residual. Fixed N needs a single-grid context.   */
                           /* Atom number, angular momentum and mu are observables (ss_obs)*/
#define SS_SID 5           /* s+id two-band superconductor (Table 1), params               */
                           /* {a1, a2, b1, b2, b3, b4, nu}: Delta_s, Delta_d, A (6 planes:  */
                           /* Re, Im Delta_s, Re, Im Delta_d, A_1, A_2), D = d - i A,       */
                           /* gradient tensor identity per band and nu diag(1, -1) between  */
                           /* them (d_{x^2-y^2}); V = a1|Ds|^2 + a2|Dd|^2 + b1|Ds|^4 +      */
                           /* b2|Dd|^4 + b3|Ds|^2|Dd|^2 + b4 (Ds^2 conj(Dd)^2 + c.c.);      */
                           /* needs |nu| < 1, b1, b2 > 0, 4 b1 b2 > (b3 - 2|b4|)^2          */

/* ---- minimisers ---- */
#define SS_METHOD_ANF 0      /* arrested Newton flow, RK4 + Eq. 4 (Sec. 3.2): the default */
#define SS_METHOD_GRADIENT 1 /* gradient descent, the first-order method Sec. 3.2 compares */
                             /* against: phi <- phi - dtau G(phi) (explicit Euler on the   */
                             /* gradient flow; chiral magnet renormalised), one launch a   */
                             /* step                                                        */

typedef struct ss_ctx ss_ctx;

/* One soliton of an initial configuration (Sec. 3.4 "model-specific ansatz"; the
 * paper gives no formula, the standard forms are used):
 *  Abelian Higgs: psi = prod_k tanh(r_k/size_k)^|charge_k| exp(i (charge_k theta_k + phase_k)),
 *                 A = sum_k charge_k tanh(r_k/size_k)^2 (-(y-y_k), x-x_k) / r_k^2.
 *  Chiral magnet and Baby Skyrme: compact skyrmion of radius R = size, vorticity m = charge,
 *                 helicity gamma = phase: n = (sin f cos(m theta + gamma),
 *                 sin f sin(m theta + gamma), cos f), f = pi (1 - r/R) for r < R,
 *                 n = e_3 outside every disc; the first disc containing a site wins.
 *                 Its lattice charge is -m.
 *  s+id: the Abelian Higgs vortex product (same windings and sizes) scaled by the
 *       uniform minimum of the potential: Delta_s = sqrt(S) x it, Delta_d = sqrt(D)
 *       e^{i phi} x it with the relative phase phi = pi/2 for b4 > 0 (else 0); A as for
 *       the Abelian Higgs model. Charge: winding of Delta_s; flux as Abelian Higgs.
 *  BEC: the Thomas-Fermi amplitude sqrt(max(0, mu - r^2/2) / g) times a vortex factor
 *       tanh(r_k/size_k)^|charge_k| exp(i (charge_k theta_k + phase_k)) per entry (an
 *       entry of charge 0 and phase 0 gives the Thomas-Fermi profile alone). At a fixed
 *       atom number N, mu = sqrt(g N / pi), the Thomas-Fermi value for N atoms (then
 *       scaled to N exactly by the refresh of the new field). */
typedef struct {
  double x, y;
  int charge;
  double size, phase;
} ss_soliton;

/* Flow status after ss_step / ss_minimise. Under SS_METHOD_GRADIENT nothing is
 * arrested: `arrests` counts the steps that raised the energy (a sign that dtau is
 * past the stability limit), `arrested` tells whether the last one did, and
 * `energy_change` is the plain difference of the two energies. Those energies are
 * summed in the working precision, so with FP32 fields the count also picks up
 * rounding noise once the per-step decrease falls below it (near convergence). */
typedef struct {
  double energy;      /* E_h of the current field as the flow sums it. FP32 kernels   */
                      /* sum it on the first field, every 16th step and the last     */
                      /* field of a run; in between it is the previous E_h plus the  */
                      /* exact change (energy_change). ss_observables: FP64.         */
  double grad_max;    /* dx dy max_I |G| of the current field: the convergence measure */
  long long steps;    /* steps taken since the fields were last set                    */
  long long arrests;  /* arrests (Eq. 4) since the fields were last set                */
  int converged;      /* grad_max < tol (ss_minimise only)                             */
  int arrested;       /* the current velocity is zeroed by a pending arrest            */
  double energy_change; /* E_h(current) - E_h(previous field) as used by the arrest     */
                        /* test, summed per site in cancellation-free form (0 if none)  */
} ss_status;

/* Observables of the current field, evaluated in FP64 arithmetic. */
typedef struct {
  double energy;       /* E_h = dx dy sum_I e                                           */
  double charge;       /* chiral magnet: Berg-Luescher lattice charge; Abelian Higgs:   */
                       /* winding of arg psi around the boundary of I                   */
  double flux;         /* Abelian Higgs: dx dy sum_I (d_1 A_2 - d_2 A_1); else 0        */
  double grad_max;     /* dx dy max_I |G|                                               */
  double grad_max_raw; /* max_I |G|                                                     */
  double norm_dev;     /* chiral magnet: max over sites of ||n| - 1|; else 0            */
  long long steps;     /* steps taken since the fields were last set                    */
  double atoms;        /* BEC: N = dx dy sum_I |psi|^2; else 0                          */
  double angular_momentum; /* BEC: dx dy sum_I Re(psi* L_z psi); else 0                 */
  double chemical_potential; /* BEC: mu in force (the given one, or the multiplier of    */
                             /* the current field at a fixed atom number); else 0         */
} ss_obs;

/* Message for the calling thread's last failed call ("" if none). Owned by the
 * library; valid until the thread's next failing call. */
const char* ss_last_error(void);

/* Library ABI version (increments on incompatible changes). */
int ss_version(void);

/* Create a context for an nx x ny grid (halo included; nx, ny >= 5) with spacings
 * dx, dy > 0 (Sec. 3.1 lattice). precision: SS_FP32, SS_FP64 or SS_FP32_PLAIN. cuda_stream: a
 * cudaStream_t borrowed for the context's lifetime, or NULL (see above). The
 * context uses the calling thread's current CUDA device. The time step is
 * dt = 0.5 min(dx, dy) (Sec. 3.1, Courant number C = 0.5). Device buffers are
 * allocated by ss_set_theory. Errors: SS_ERR_ARG, SS_ERR_CUDA, SS_ERR_NOMEM. */
int ss_create_grid(ss_ctx** out, int nx, int ny, double dx, double dy, int precision, void* cuda_stream);

/* Select the theory and its couplings (Sec. 3.1 "theory-specific parameters packed
 * into device arrays"; Table 1; Eq. 5). params is a host array of n_params
 * doubles: Abelian Higgs {lambda, u} (u defaults to 1 if n_params == 1); chiral
 * magnet {J, D, K, h, dmi_type, mu_d} (dmi_type and mu_d default to 0); Baby
 * Skyrme {kappa, mu, nu} (nu defaults to 0 if n_params == 2); BEC {g, Omega, mu}
 * with g > 0 (the BEC's charge observable is 0: see atoms, angular_momentum); s+id
 * {a1, a2, b1, b2, b3, b4, nu} (see SS_SID for the constraints).
 * Allocates the device buffers; previous fields are discarded.
 * Errors: SS_ERR_ARG (unknown theory, bad n_params, J <= 0), SS_ERR_NOMEM, SS_ERR_CUDA. */
int ss_set_theory(ss_ctx* ctx, int theory, const double* params, int n_params);

/* Set the fields to the ansatz of n >= 1 solitons (host array, copied), evaluated
 * in FP64 on the device and rounded to the context precision; the halo receives the
 * same formula and is then frozen. Velocity v = 0 (flow from rest, Sec. 3.2).
 * Errors: SS_ERR_STATE (no theory), SS_ERR_ARG (n < 1, size <= 0), SS_ERR_CUDA. */
int ss_init_ansatz(ss_ctx* ctx, const ss_soliton* solitons, int n);

/* Copy a caller field array [C][ny][nx] (context precision) into the context,
 * halo included, and restart the flow from rest (v = 0, no pending arrest): the
 * resume step of a checkpoint. Errors: SS_ERR_STATE, SS_ERR_ARG (NULL), SS_ERR_CUDA. */
int ss_set_fields(ss_ctx* ctx, const void* fields, int is_device);

/* Copy the current field [C][ny][nx] (context precision) out to the caller.
 * Errors: SS_ERR_STATE, SS_ERR_ARG, SS_ERR_CUDA. */
int ss_get_fields(ss_ctx* ctx, void* fields, int is_device);

/* ss_batch_autotune for a single-grid context (see there); the context's field is
 * kept, the flow restarts from rest. */
int ss_autotune(ss_ctx* ctx, int trial_steps, int* choice);
/* ss_batch_set_method for a single-grid context (needs ss_set_theory first). */
int ss_set_method(ss_ctx* ctx, int method, double step_factor);
/* ss_batch_set_launch for a single-grid context. */
int ss_set_launch(ss_ctx* ctx, int tile_shape, const int* blocks);

/* SS_FP32 contexts: copy the rounding remainder of the current field [C][ny][nx]
 * (float), so that value + remainder (summed in FP64) is the field the flow holds;
 * other precisions write zeros. Errors as ss_get_fields. */
int ss_get_remainder(ss_ctx* ctx, void* remainder, int is_device);

/* Copy the current velocity phi-dot [C][ny][nx] out, with a pending arrest (Eq. 4)
 * applied (zeros if the last step raised the energy; always zeros under
 * SS_METHOD_GRADIENT). Errors as ss_get_fields. */
int ss_get_velocity(ss_ctx* ctx, void* velocity, int is_device);

/* Euler-Lagrange force G of the current field (the right-hand side of Eq. 3 up to
 * sign; chiral magnet tangent-projected), [C][ny][nx], zero on the halo, in the
 * context precision. Optionally returns E_h and dx dy max|G| (may be NULL).
 * Errors: SS_ERR_STATE, SS_ERR_ARG, SS_ERR_CUDA. */
int ss_force(ss_ctx* ctx, void* force, int is_device, double* energy, double* grad_max);

/* Take n_steps >= 0 arrested-Newton-flow RK4 steps (Sec. 3.2, Eq. 3, Eq. 4), or
 * gradient-descent steps after ss_set_method(SS_METHOD_GRADIENT). The
 * energy of each new field is reduced on the device and compared with the previous
 * one there; the host is not involved between steps. out (may be NULL) receives
 * the status of the resulting field. Errors: SS_ERR_STATE, SS_ERR_ARG,
 * SS_ERR_NONFINITE (flow stopped at the first non-finite energy/force), SS_ERR_CUDA. */
int ss_step(ss_ctx* ctx, int n_steps, ss_status* out);

/* Run the flow until dx dy max_I |G| < tol (checked before every step) or
 * max_steps steps have been taken in this call. Steps run in CUDA-graph chunks;
 * the host polls one small status record per chunk. With FP32 fields the flow's
 * own residual is FP32 arithmetic, so the verdict is the FP64 evaluation of the
 * stored field (value + remainder, as ss_observables): while that is not below
 * tol, the flow takes further rounds of steps (1/64 of the steps taken so far, 8 to
 * 512 per round) within the same max_steps, and is judged again. Returns SS_OK if converged, SS_ERR_NOT_CONVERGED if
 * max_steps was reached, SS_ERR_NONFINITE, or another error. out (may be NULL)
 * receives the final status in every case (its grad_max is the flow's own). */
int ss_minimise(ss_ctx* ctx, double tol, long long max_steps, ss_status* out);

/* Observables of the current field (Sec. 2: "GPU-resident evaluation of
 * observables"; Sec. 3.3 reductions), in FP64 arithmetic with compensated sums.
 * Errors: SS_ERR_STATE, SS_ERR_ARG (NULL), SS_ERR_CUDA. */
int ss_observables(ss_ctx* ctx, ss_obs* out);

/* Tracing: take n_steps (1..4096) flow steps exactly as ss_step does, but with
 * direct launches bracketed by CUDA events on the context stream, and return the
 * mean device duration in milliseconds of the two kernels of a step:
 * ms_out[0] = pass 1 (RK stages 1-2 with the energy / residual / energy-change
 * reductions and the on-device arrest decision of Eq. 4), ms_out[1] = pass 2 (RK
 * stages 3-4 and the RK4 combination). Under SS_METHOD_GRADIENT ms_out[0] is the
 * descent kernel (one per step) and ms_out[1] = 0. The steps advance the flow.
 * Errors: SS_ERR_STATE, SS_ERR_ARG, SS_ERR_CUDA, SS_ERR_NONFINITE. */
int ss_profile_stages(ss_ctx* ctx, int n_steps, float* ms_out);

/* Release every device and host resource of the context (NULL is a no-op). */
int ss_destroy(ss_ctx* ctx);

/* ---- batches ---------------------------------------------------------------
 * Many independent relaxations (uneven grid sizes, spacings, couplings and initial
 * solitons; one theory and one precision) advanced together: every flow kernel
 * launch covers the tiles of all problems, each problem keeps its own step count,
 * arrest test (Eq. 4), convergence test and buffers, and stops on its own. Steps
 * run in CUDA graphs of 32 steps; the host polls one counter of still-running
 * problems per graph. Semantics per problem are those of ss_step / ss_minimise. */
typedef struct ss_batch ss_batch;

/* One problem of a batch. params / solitons are host arrays, copied at creation. */
typedef struct {
  int nx, ny;            /* grid incl. the width-2 halo, >= 5 each              */
  double dx, dy;         /* spacings > 0; dt = 0.5 min(dx, dy)                  */
  const double* params;  /* couplings as for ss_set_theory                      */
  int n_params;
  const ss_soliton* solitons; /* initial ansatz (ss_init_ansatz), n_solitons >= 1 */
  int n_solitons;
} ss_batch_item;

/* Create a batch of n >= 1 problems of `theory` in `precision`, each initialised
 * from its ansatz, at rest. cuda_stream as for ss_create_grid.
 * Two forms need a single-grid context and are rejected here (SS_ERR_ARG): the chiral
 * magnet with demagnetisation (mu_d > 0; its Poisson solve is per grid) and the BEC at a
 * fixed atom number (N > 0; its refresh reduces over one grid).
 * Errors: SS_ERR_ARG (message names the item), SS_ERR_NOMEM, SS_ERR_CUDA. */
int ss_batch_create(ss_batch** out, int theory, int precision, const ss_batch_item* items, int n, void* cuda_stream);

/* Number of problems of the batch (0 for NULL). */
int ss_batch_size(ss_batch* batch);

/* n_steps more flow steps for every problem that has not stopped. per_item (n
 * entries, may be NULL) receives every problem's status.
 * Errors: SS_ERR_ARG, SS_ERR_NONFINITE (some problem stopped non-finite), SS_ERR_CUDA. */
int ss_batch_step(ss_batch* batch, int n_steps, ss_status* per_item);

/* Flow every problem until its own dx dy max|G| < tol or max_steps more steps.
 * Returns SS_OK when all converged, SS_ERR_NOT_CONVERGED when some did not,
 * SS_ERR_NONFINITE when some stopped non-finite; per_item (may be NULL) tells which. */
int ss_batch_minimise(ss_batch* batch, double tol, long long max_steps, ss_status* per_item);

/* Copy the current field of problem `item` ([C][ny][nx], batch precision) out. */
int ss_batch_get_fields(ss_batch* batch, int item, void* fields, int is_device);

/* Replace the field of problem `item` (same layout and precision; halo included, the
 * halo values become its Dirichlet data) and restart its flow from rest with a
 * fresh step count, as ss_set_fields does for a single grid. */
int ss_batch_set_fields(ss_batch* batch, int item, const void* fields, int is_device);

/* Autotuner (no counterpart in the paper): times every tile shape of the flow kernels
 * (FP32: 32 x 16 or 32 x 32 sites, FP64: 32 x 8 or 32 x 16) and every grid size of
 * each pass (1 .. occupancy blocks per SM x SMs) with CUDA events over trial_steps
 * (1..1000) flow steps of the batch's own problems, and keeps the fastest. Every
 * problem is then reset to the field it had at the call, at rest (v = 0), with its
 * step count back at 0. choice (may be NULL) receives {tile shape 0|1, pass-1 blocks,
 * pass-2 blocks}. Uses a temporary device copy of the fields.
 * Errors: SS_ERR_ARG, SS_ERR_NOMEM, SS_ERR_CUDA. */
int ss_batch_autotune(ss_batch* batch, int trial_steps, int* choice);

/* Set the flow launch by hand (what ss_batch_autotune chooses): tile_shape 0 (small)
 * or 1 (large, the default); blocks = {pass-1 grid, pass-2 grid}, or NULL for each
 * pass's occupancy x SMs (capped by the tile count). Fields and flow state are kept.
 * Under SS_METHOD_GRADIENT blocks[0] is the grid of the descent kernel and
 * blocks[1] is ignored; ss_batch_autotune likewise times only that kernel and
 * returns {tile shape, descent blocks, 0}.
 * Errors: SS_ERR_ARG, SS_ERR_CUDA. */
int ss_batch_set_launch(ss_batch* batch, int tile_shape, const int* blocks);

/* Select the minimiser of every problem (SS_METHOD_ANF, the default, or
 * SS_METHOD_GRADIENT). step_factor sets gradient descent's step as a fraction of
 * the Euler stability limit of the Eq. 2 Laplacian, dtau = step_factor * (3/8) /
 * (1/dx^2 + 1/dy^2) per problem; it must be in (0, 1], and <= 0 selects 0.8. (The
 * limit is 2 / lambda_max with lambda_max = (16/3)(1/dx^2 + 1/dy^2), the stencil's
 * largest eigenvalue; the couplings' own terms shift it by O(dx^2). For SS_BEC,
 * lambda_max also carries bounds of the trap, r_max^2, the interaction, 4 |mu|,
 * and the rotation, 2 |Omega| r_max 1.3722 / min(dx, dy), over the grid.) Every problem
 * whose fields are set restarts from its current field at rest, with its step
 * count and flow record cleared; tile shape and grids are kept. Descent takes one
 * kernel launch per step: it evaluates E_h, dx dy max|G| and -G of the current field
 * (so ss_force stays valid), writes the next field, and stops as ss_minimise
 * describes. Errors: SS_ERR_ARG, SS_ERR_CUDA. */
int ss_batch_set_method(ss_batch* batch, int method, double step_factor);

/* Observables of problem `item`, as ss_observables. */
int ss_batch_observables(ss_batch* batch, int item, ss_obs* out);

/* Release the batch (NULL is a no-op). */
int ss_batch_destroy(ss_batch* batch);

/* Observables of a caller-owned device field without allocating anything.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc -- code whose device memory belongs to a framework's caching
 * allocator or to a fixed arena that must account for every byte, and code where
 * an allocation would implicitly synchronize the device or could fail because the
 * device memory is already fully reserved. It computes exactly what ss_observables
 * computes (same kernels, same FP64 compensated reductions) for the field at
 * `fields`, without a context, and calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 *  theory, params, n_params: as ss_set_theory (validated by the same rules), except
 *             that the two forms that need a context's state are rejected:
 *             demagnetisation (mu_d > 0) and the BEC at a fixed atom number (N > 0).
 *  fields:    device pointer, [C][ny][nx] planes of the given precision (float for
 *             SS_FP32 and SS_FP32_PLAIN, double for SS_FP64), halo included. Read
 *             only. For SS_FP32 this is the value plane alone (no remainder).
 *  nx, ny, dx, dy: as ss_create_grid; nx, ny <= 65536 and nx * ny <= 2^31, larger
 *             grids are rejected with SS_ERR_ARG.
 *  out:       device pointer to 6 doubles, written with {energy, charge, flux,
 *             grad_max, grad_max_raw, norm_dev} (the ss_obs fields of the same names).
 *  cuda_stream: the stream to run on (NULL = legacy default stream). The call only
 *             enqueues work: `out` is valid once that stream's work has completed.
 *
 * Scratch: the reduction's block partials, arrival counter and result record live
 * in one file-scope device array of 128.25 KB (at most 2048 reducing blocks; the
 * kernel strides over tiles, so every allowed grid fits). Every GPU that loads the
 * library holds this array until the process exits. All calls on a device share
 * it and it keeps the last call's contents: each call clears the counter it needs
 * zeroed, but calls whose GPU work overlaps (different streams or host threads
 * without ordering between them) race on it and must be serialized by the caller.
 * Every call looks up the array's device address (cudaGetSymbolAddress) on the
 * caller's current device, so no address outlives a device reset. The first call
 * on a device also loads the library's device code there: make that first call
 * before any stream capture.
 *
 * Errors: SS_ERR_ARG (NULL pointers, sizes, spacings, theory, params), SS_ERR_CUDA. */
int ss_observables_noalloc(int theory, const double* params, int n_params, const void* fields, int nx, int ny,
                           double dx, double dy, int precision, double* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SOLITON_H */
