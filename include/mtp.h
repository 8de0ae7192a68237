/*
 * mtp.h -- C ABI of the GB300 Moment Tensor Potential library (libmtp.so).
 *
 * Method: "The MLIP package: Moment Tensor Potentials with MPI and Active Learning",
 * arXiv:2007.08555, Sec. 2.  Every entry point cites the passage that defines what it computes.
 *
 * Conventions (all entry points)
 *   - Units: Angstrom, eV, eV/Angstrom.  The virial W = -dE/d(eps) (eV, extensive, row-major
 *     3x3) is returned instead of the stress; stress in GPa is -W / volume * 160.21766.
 *   - A cell is given by its three lattice vectors as rows: cell[3*k + d] = component d of a_k.
 *     Positions need not lie inside the cell (they are used as given for r_ij = x_j + s H - x_i).
 *   - Species indices are 0 .. n_species-1; anything else is MTP_EINVAL.
 *   - Batches are CSR over configurations: the atoms of configuration k are
 *     cfg_off[k] .. cfg_off[k+1]-1 (cfg_off[0] = 0, non-decreasing).
 *   - Pointers are device pointers unless flags contains MTP_HOST_MEMORY, in which case every
 *     array argument of that call is host memory (pinned memory makes the copies asynchronous).
 *     The caller owns every array argument; the library owns the model, its device scratch and
 *     its active set.  Output arrays that may be NULL are skipped when NULL.
 *   - Calls are ordered on the CUDA stream passed as `stream` (a cudaStream_t; NULL = the
 *     legacy default stream).  Without MTP_ASYNC a call synchronises that stream before it
 *     returns and reports device-detected errors in its status; with MTP_ASYNC it returns after
 *     enqueueing and device-detected errors are reported by the next mtp_sync().
 *   - No C++ exception crosses this boundary; every call returns an mtp_status.
 *   - A model is not thread-safe: calls on one model must not overlap (they share scratch).
 */
#ifndef MTP_H
#define MTP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mtp_model mtp_model;

typedef enum {
    MTP_OK = 0,
    MTP_EINVAL = 1,        /* invalid argument (size, species index, level, null pointer) */
    MTP_ENOMEM = 2,        /* device allocation failed */
    MTP_ECUDA = 3,         /* a CUDA runtime call failed */
    MTP_EOVERFLOW = 4,     /* an atom has more neighbours than the list capacity */
    MTP_ESINGULAR = 5,     /* the active-set matrix is singular */
    MTP_ETIMEOUT = 6,      /* an iteration limit was reached (MaxVol swaps) */
    MTP_ENOACTIVESET = 7,  /* grades requested but no active set has been built */
    MTP_EUNSUPPORTED = 8   /* valid request that this build does not support */
} mtp_status;

typedef enum {
    MTP_FP64 = 0,    /* every step in double precision */
    MTP_FP32 = 1,    /* pair geometry, radial basis, moments, contractions and adjoint in float;
                        per-configuration energy and virial sums in double */
    MTP_FP32_TC = 2  /* MTP_FP32, and the grade product b A^-1 (Sec. 2.3) on the tensor cores: BF16
                        digit products accumulated in FP32 (exact group sums), combined exactly;
                        error comparable to a double-precision product (see mtp_grade) */
} mtp_precision;

enum {
    MTP_HOST_MEMORY = 1,      /* array arguments are host pointers */
    MTP_ASYNC = 2,            /* do not synchronise the stream before returning */
    MTP_REUSE_NEIGHBORS = 4   /* reuse the neighbour list of the previous call on this model
                                 (same atoms, cfg_off and cells; positions may have moved) */
};

/* Human-readable name of a status code (static storage). */
const char* mtp_status_str(mtp_status s);

/*
 * Create a potential (Sec. 2.1).
 *   lev_max     maximum level of a basis function, Eq. 5 / Eq. 6; even, 2 <= lev_max <= 20
 *               (basis levels are always even, an odd value is rounded down).
 *   n_species   number of atomic types S (1..8).
 *   n_radial    N_Q, the number of radial basis functions Q_b of Eq. 4 (1..16).
 *   r_min, r_cut  the interval [R_min, R_cut] of the Chebyshev polynomials, Eq. 4; 0 <= r_min < r_cut.
 *   xi          host array [m] of the linear coefficients of Eq. 2 in the order of
 *               mtp_level_table(), or NULL for zeros.
 *   c           host array [S][S][N_mu][N_Q] of the radial coefficients c_{mu,z_i,z_j}^{(b)} of
 *               Eq. 3, first index z_i (the central atom), or NULL for zeros.
 *   prec        MTP_FP64, MTP_FP32 or MTP_FP32_TC.
 *   out         receives the model; release it with mtp_destroy().
 * Uses the current CUDA device.  Returns MTP_EINVAL for out-of-range arguments.
 */
mtp_status mtp_create(int lev_max, int n_species, int n_radial, double r_min, double r_cut, const double* xi,
                      const double* c, mtp_precision prec, mtp_model** out);

/* Release the model and all device memory it owns (NULL is allowed). */
void mtp_destroy(mtp_model* model);

/* m, the number of basis functions B_alpha (length of xi), Eq. 2. */
int mtp_basis_count(const mtp_model* model);
/* N_mu, the number of radial functions f_mu (Eq. 3): floor((lev_max - 2) / 4) + 1. */
int mtp_radial_count(const mtp_model* model);
/* C, the number of symmetric moment-tensor components stored per atom (Sec. 2.1). */
int mtp_moment_count(const mtp_model* model);

/*
 * The canonical level table: the basis of Sec. 2.1 as loopless multigraphs (node = moment
 * M_{mu,nu}, edge = one contracted index pair; a basis function is the product of its connected
 * components).  Layout (int32): [m, then per basis function: level, n_components, then per
 * component: n, mu_0, nu_0, ..., mu_{n-1}, nu_{n-1}, A[0][1], A[0][2], ..., A[n-2][n-1]].
 * A component's node order is the one giving the lexicographically smallest such code;
 * components are ordered by (level, n, code), basis functions by (level, total number of
 * moments, ascending component numbers).  Writes min(cap, len) ints to buf (buf may be NULL)
 * and the full length to *len.
 */
mtp_status mtp_level_table(const mtp_model* model, int32_t* buf, size_t cap, size_t* len);

/* Replace theta = {xi, c} (host arrays, layouts as in mtp_create; NULL keeps the old value). */
mtp_status mtp_set_params(mtp_model* model, const double* xi, const double* c);

/* Skin added to R_cut when neighbour lists are built (default 0).  With a skin > 0 the build also
 * keeps the positions, and an evaluation with MTP_REUSE_NEIGHBORS (same atoms, configurations and
 * cells) refreshes r_ij = r0_ij + (u_j - u_i) from the displacements u since the build instead of
 * searching again; pairs beyond R_cut contribute nothing (Q_b = 0 there, Eq. 4).  The caller must
 * rebuild before any atom has moved by skin / 2. */
mtp_status mtp_set_skin(mtp_model* model, double skin);

/* Threads per atom in the pair kernels: `moments` for the moment accumulation (Eq. 5), `pairs` for
 * the pair gradients, the force gather and the loss-gradient kernels; each 1, 2, 4 or 8, or 0
 * (default) to choose per call from the atom count.  A tuning knob without a counterpart in the paper: results agree to
 * rounding whatever the choice (summation order changes).  Other values are MTP_EINVAL. */
mtp_status mtp_set_threads_per_atom(mtp_model* model, int moments, int pairs);

/*
 * Autotuner of the batched launch (no counterpart in the paper): times the evaluation (neighbour
 * search + E, F, W) of this batch for every lanes-per-atom choice of the moment kernel and of the
 * pair-gradient, gather and loss-gradient kernels ({1, 2, 4, 8} each; median of five graph
 * replays after three untimed calls) and records the fastest for the size class of the batch:
 * (lev_max, S, N_Q, precision, floor(log2 n_atoms), SM count), shared by every model of the process.
 * Models whose mtp_set_threads_per_atom() setting is 0 (the default) use the recorded choice for
 * batches of that class, and the built-in heuristic for others.  Device arrays (batch layout of
 * mtp_eval_batch); best_moments, best_pairs and times_ms ([16] in ms, index 4 * log2(moments) +
 * log2(pairs)) are host pointers and may be NULL.  Synchronous; the model's own setting is kept.
 */
mtp_status mtp_autotune(mtp_model* model, int n_cfg, int n_atoms, const int32_t* cfg_off, const double* pos,
                        const int32_t* types, const double* cells, int* best_moments, int* best_pairs,
                        double* times_ms, void* stream);

/* Capacity of the per-atom neighbour list (default 128).  MTP_EOVERFLOW reports the largest
 * count seen through *max_seen of mtp_last_neighbor_max(). */
mtp_status mtp_set_neighbor_capacity(mtp_model* model, int cap);
int mtp_last_neighbor_max(const mtp_model* model);

/*
 * Neighbourhoods (Sec. 2.1, Eq. 1): for each atom i every (j, s), s an integer image shift, with
 * |x_j + s H - x_i| < r_cut (strict), excluding (i, s = 0); skin adds to r_cut.  The decision is
 * taken in double precision as d_k = (x_j[k] + ((s_0 H_0k + s_1 H_1k) + s_2 H_2k)) - x_i[k],
 * r^2 = (d_0^2 + d_1^2) + d_2^2, without fused multiply-adds.  Lists are sorted by (j, s_0, s_1, s_2).
 * Outputs (CSR over atoms): counts[n_atoms]; then, if nbr_j is not NULL, nbr_j[P], nbr_s[P][3] and
 * r_ij[P][3] (double) with P = sum(counts) <= cap_pairs (else MTP_EOVERFLOW, counts still written).
 * Shifts are limited to |s_k| <= 127 (positions more than ~120 cells outside their cell: MTP_EINVAL).
 */
mtp_status mtp_neighbors(mtp_model* model, int n_cfg, int n_atoms, const int32_t* cfg_off, const double* pos,
                         const double* cells, double skin, int32_t* counts, int32_t* nbr_j, int32_t* nbr_s,
                         double* r_ij, int64_t cap_pairs, int flags, void* stream);

/*
 * Energy, forces and virial of a batch of periodic configurations (Sec. 2.1, Eqs. 1-4):
 *   E_k = sum_i V(n_i), V(n_i) = sum_alpha xi_alpha B_alpha(n_i),  F = -dE/dx,  W = -dE/d(eps).
 * Inputs: n_cfg configurations, n_atoms atoms in total, cfg_off[n_cfg+1], pos[n_atoms][3],
 * types[n_atoms], cells[n_cfg][9].
 * Outputs (each may be NULL): energy[n_cfg], forces[n_atoms][3], virial[n_cfg][9],
 *   site_energy[n_atoms] (V(n_i)), b_rows[n_cfg][m] (b_alpha(cfg) = sum_i B_alpha(n_i), Eq. 13),
 *   b_atoms[n_atoms][m] (B_alpha(n_i)),
 *   grade_cfg[n_cfg] (gamma = max_j |(b A^-1)_j|, Sec. 2.3) and grade_atom[n_atoms]
 *   (max_j |(B(n_i) A^-1)_j|), both against the active set of mtp_select_active_set()
 *   (MTP_ENOACTIVESET without one).
 * flags: MTP_HOST_MEMORY, MTP_ASYNC, MTP_REUSE_NEIGHBORS.
 */
mtp_status mtp_eval_batch(mtp_model* model, int n_cfg, int n_atoms, const int32_t* cfg_off, const double* pos,
                          const int32_t* types, const double* cells, double* energy, double* forces, double* virial,
                          double* site_energy, double* b_rows, double* b_atoms, double* grade_cfg,
                          double* grade_atom, int flags, void* stream);

/* One configuration: mtp_eval_batch with n_cfg = 1 (cell[9], virial[9]). */
mtp_status mtp_eval(mtp_model* model, int n_atoms, const double* pos, const int32_t* types, const double* cell,
                    double* energy, double* forces, double* virial, double* site_energy, double* grade_cfg,
                    double* grade_atom, int flags, void* stream);

/*
 * Active set by MaxVol (Sec. 2.3, Eq. 13; Goreinov et al. 2010).  Chooses m of the n_rows >= m rows of
 * the tall matrix b_rows [n_rows][m] (double) so that |det A| of the m x m submatrix cannot grow by
 * exchanging one row: start from the pivot rows of Gaussian elimination with partial pivoting, then
 * repeatedly let the row and column of the largest |c| of C = B A^-1 swap in, while it exceeds 1 + 1e-3
 * (ties: smallest row, then smallest column), at most 100 m swaps.  Columns are first scaled by
 * 1 / max |column|, which changes neither C nor the selection but conditions the arithmetic.  A and A^-1 (double) stay in the
 * model for grades.  selected[m] receives the chosen row indices (position j = row of A), n_swaps the
 * number of exchanges and max_grade the final max |C| (each may be NULL).  MTP_HOST_MEMORY: b_rows and
 * selected are host arrays.  Synchronous.  MTP_ESINGULAR: B has rank < m; MTP_ETIMEOUT: swap limit.
 */
mtp_status mtp_select_active_set(mtp_model* model, int n_rows, const double* b_rows, int32_t* selected, int* n_swaps,
                                 double* max_grade, int flags, void* stream);

/*
 * MaxVol active-set selection that allocates nothing (the paper has no counterpart: this is a
 * library service).  For callers that must not allocate device memory -- a time-step loop where a
 * cudaMalloc could synchronise the device and stall other work, or an application whose device
 * memory is entirely owned by its own pool -- it runs the algorithm of mtp_select_active_set() with
 * all scratch in one fixed array built into the library (4 MiB, held on every GPU that loads the
 * library until the process exits).  Limit: the scratch layout must fit that array of 524,288
 * doubles, i.e.  2 n m + max(n m, 2 m^2) + 2 m^2 + 3 m + n + ceil((n + m + 2) / 2) + 1 <= 524,288
 * with n = n_rows (n <= 1421 at m = 116, n <= 1671 at m = 100; n = 2 m fits up to m = 255, so the
 * lev_max-20 basis, m = 460, does not fit);
 * larger sizes return MTP_EINVAL before any work.
 * Inputs and outputs are the caller's device arrays: b_rows [n_rows][m] (double), selected [m]
 * (int32, the chosen row of each position), a_inv [m][m] (double, may be NULL); n_swaps is a host
 * pointer (may be NULL).  It needs no model and keeps no active set.  The first call on each device
 * looks up the array's device address; make that first call before any stream capture.  All calls
 * share the array, which keeps the last call's contents: calls that overlap on the GPU race.
 * Synchronous on `stream`.  MTP_ESINGULAR / MTP_ETIMEOUT as for mtp_select_active_set().
 */
mtp_status mtp_select_active_set_noalloc(int n_rows, int m, const double* b_rows, int32_t* selected, double* a_inv,
                                         int* n_swaps, void* stream);

/*
 * Active-set update from candidate configurations (Sec. 2.3: the selected, extrapolative
 * configurations enter the training set where they raise |det A|; at most m of them, however many
 * were selected).  MaxVol on the stacked matrix [A; cand_rows] (cand_rows [n_cand][m] double, b rows
 * of the candidates) starting from the current active set (rows 0 .. m-1), with the swap rule,
 * tolerance and iteration limit of mtp_select_active_set(); the result replaces the model's A and
 * A^-1.  Outputs (host, each may be NULL): entered [m] the candidate indices now in the active set
 * (ascending, *n_entered of them), rows [m] the final active set as indices into the stacked matrix
 * (position j = row j of the new A), n_swaps.  cand_rows is device memory unless MTP_HOST_MEMORY.
 * Synchronous.  MTP_ENOACTIVESET without an active set; MTP_ESINGULAR / MTP_ETIMEOUT as for
 * mtp_select_active_set() (the active set is then dropped).
 */
mtp_status mtp_select_add(mtp_model* model, int n_cand, const double* cand_rows, int32_t* entered, int* n_entered,
                          int32_t* rows, int* n_swaps, int flags, void* stream);

/*
 * Kind of extrapolation grade (Sec. 2.3): 0 (default) the linear criterion, rows b(cfg) of width m;
 * 1 the nonlinear criterion, where the rows are the Jacobian dE(cfg)/dtheta over the parameters
 * theta = [xi (m), c (S, S, N_mu, N_Q) in C order].  The full Jacobian rows satisfy exact linear
 * relations (E is homogeneous in each radial block c[:, :, mu, :], Euler's theorem), so no square
 * submatrix of them is invertible; cols (host, n_cols ascending indices into theta) selects an
 * independent set of parameter columns, e.g. by a column-pivoted QR of training rows; NULL takes
 * all m + S^2 N_mu N_Q.  The active set (mtp_select_active_set, mtp_select_add, mtp_set_active_set,
 * mtp_get_active_set, mtp_grade, model files) then has width n_cols (mtp_grade_width(),
 * mtp_grade_columns()); changing the kind drops the installed active set.  In the nonlinear kind,
 * rows come from mtp_jacobian_rows() and are graded with mtp_grade(); mtp_eval_batch's grades,
 * mtp_md_select and grade-checked relaxations return MTP_EUNSUPPORTED.  MTP_EINVAL for columns
 * out of range or not ascending.
 */
mtp_status mtp_set_grade_kind(mtp_model* model, int nonlinear, int n_cols, const int32_t* cols);
int mtp_grade_width(const mtp_model* model);
mtp_status mtp_grade_columns(const mtp_model* model, int32_t* cols /* host [mtp_grade_width()] */);

/*
 * Jacobian rows of the nonlinear criterion (Sec. 2.3) for a batch (layout of mtp_eval_batch, device
 * arrays): rows [n_cfg][mtp_grade_width()] (double, device), the columns selected by
 * mtp_set_grade_kind() of [b(cfg_k), dE_k/dc] with b(cfg_k) = sum_i B(n_i) = dE_k/dxi (Eq. 2) and
 * dE_k/dc from the adjoint kernels of mtp_param_grad, summed per configuration in double precision.
 * In the linear kind the rows are [b(cfg_k), dE_k/dc] in full.  Flags: MTP_ASYNC.
 */
mtp_status mtp_jacobian_rows(mtp_model* model, int n_cfg, int n_atoms, const int32_t* cfg_off, const double* pos,
                             const int32_t* types, const double* cells, double* rows, int flags, void* stream);

/* Install an active set given its w x w matrix A (host, row-major; rows = b (or Jacobian rows) of the
 * active configurations; w = mtp_grade_width());
 * A^-1 is computed on the device.  MTP_ESINGULAR if A is singular. */
mtp_status mtp_set_active_set(mtp_model* model, const double* A);

/* Copy out A, A^-1 (host [m][m], may be NULL) and the selected row indices (host [m], -1 when A was set
 * directly; may be NULL).  MTP_ENOACTIVESET without an active set. */
mtp_status mtp_get_active_set(const mtp_model* model, double* A, double* A_inv, int32_t* rows);

/*
 * Write the model to a text file (the paper has no counterpart: a library service; the MLIP
 * package's own .mtp format is not used): lev_max, S, N_Q, R_min, R_cut, precision, skin,
 * neighbour-list capacity, threads per atom, theta = {xi, c} and, when one is installed, the active
 * set (A, A^-1 and its row indices).  Doubles are written with 17 significant digits, so every value
 * reads back to the same bits.  Synchronous (reads A from the device).  MTP_EINVAL if the file cannot
 * be written.
 */
mtp_status mtp_save(const mtp_model* model, const char* path);

/*
 * Create a model from a file written by mtp_save() on the current CUDA device.  The whole file is
 * read and checked before any device work: a missing or malformed file, a wrong format version,
 * counts that do not match lev_max / S / N_Q, or non-finite values give MTP_EINVAL and *out = NULL.
 * The active set is installed as saved (A^-1 is not recomputed), so grades match the saved model bit
 * for bit.
 */
mtp_status mtp_load(const char* path, mtp_model** out);

/* Extrapolation grade of arbitrary rows (Sec. 2.3): gamma[r] = max_j |(b_r A^-1)_j| for b_rows
 * [n_rows][m] (double).  Device arrays unless MTP_HOST_MEMORY.  MTP_FP64 and MTP_FP32 models form
 * the product in double precision; MTP_FP32_TC models on the tensor cores: with column scaling
 * D = 2^e (A D columns of maximum in [1/2, 1)), rows of b D and columns of G = (A D)^-1 rounded to
 * 56-bit grids relative to their largest entries 2^E_r and 2^F_j, split into 8 base-128 BF16
 * digits, digit products summed exactly in FP32 and combined exactly in integers; the error of
 * c_rj is about 1e-15 2^(E_r + F_j) and gamma is rounded to float (2^-24 relative).  A row holding
 * NaN or inf has gamma = +inf in every precision.  m <= 480 for MTP_FP32_TC. */
mtp_status mtp_grade(mtp_model* model, int n_rows, const double* b_rows, double* gamma, int flags, void* stream);

/*
 * Training loss and its exact gradient in theta = {xi, c} (Sec. 2.2, Eqs. 7, 11, 12):
 *   L = sum_k s_e w_e (E_k - e_ref_k)^2 + s_f w_f sum_i |F_i - f_ref_i|^2 + s_s w_s |W_k - w_ref_k|_F^2
 * with the per-configuration scalings of the paper, scaling = 0 "molecules" (Eq. 7: 1, 1, 1),
 * 1 "structures" (Eq. 11: 1/N^2, 1/N, 1/N^2), 2 "vibrations" (Eq. 12: 1/N, 1, 1/N); the stress
 * term uses the virial W (eV, extensive).  The batch layout is that of mtp_eval_batch; e_ref [n_cfg],
 * f_ref [n_atoms][3], w_ref [n_cfg][9].  Outputs: loss [1], d_xi [m], d_c [S][S][N_mu][N_Q] (each may
 * be NULL; with both d_xi and d_c NULL only the evaluation and the loss run).  The force and stress terms are obtained as the derivative of the pair gradients along
 * the residual displacements (the mixed second derivative), recomputed rather than stored.
 * Device arrays unless MTP_HOST_MEMORY.  Gradient sums are accumulated in double precision.
 */
mtp_status mtp_param_grad(mtp_model* model, int n_cfg, int n_atoms, const int32_t* cfg_off, const double* pos,
                          const int32_t* types, const double* cells, const double* e_ref, const double* f_ref,
                          const double* w_ref, double w_e, double w_f, double w_s, int scaling, double* loss,
                          double* d_xi, double* d_c, int flags, void* stream);

/*
 * Velocity-Verlet molecular dynamics of one periodic configuration with this potential (the paper
 * runs MD through LAMMPS, Sec. 5; this is the data-parallel step itself).  pos and vel ([n][3]
 * double, Angstrom and Angstrom/fs, device) are advanced in place by n_steps steps of dt fs;
 * masses [S] (host, amu).  Requires mtp_set_skin() > 0: the neighbour list is rebuilt when an atom
 * has moved more than skin / 2 since the last build, otherwise refreshed.  e_pot and e_kin (host,
 * [n_steps + 1], eV, step 0 = initial state) and n_rebuilds (host) may be NULL.  Energies and the
 * kinetic sum are accumulated in double precision; forces are the model's precision.
 */
mtp_status mtp_md_run(mtp_model* model, int n_atoms, double* pos, double* vel, const int32_t* types,
                      const double* cell, const double* masses, double dt, int n_steps, double* e_pot,
                      double* e_kin, int* n_rebuilds, int flags, void* stream);

/*
 * Velocity-Verlet MD with active selection (Sec. 2.3, the two-threshold scheme): mtp_md_run(), and
 * the extrapolation grade gamma of the configuration at every step, the starting one included
 * (gamma = max_j |(b A^-1)_j|, b = sum_i B(n_i), against the installed active set).  A step with
 * gamma > gamma_select is selected: its positions are copied into the device ring buffer
 * ring_pos [ring_capacity][n][3] (slot = count mod ring_capacity, so the latest frames are kept)
 * and its step and grade into the host arrays ring_steps, ring_gamma [ring_capacity].  The run
 * stops at the first step with gamma >= gamma_break (that step is selected too); pos and vel then
 * hold that configuration.  n_selected (all selections, including overwritten ones), stop_step
 * (-1 if the run completed), gammas [n_steps + 1], e_pot and e_kin ([n_steps + 1], filled up to
 * the last step run) are host pointers and may be NULL.  Requires 0 <= gamma_select < gamma_break
 * and an active set (MTP_ENOACTIVESET).
 */
mtp_status mtp_md_select(mtp_model* model, int n_atoms, double* pos, double* vel, const int32_t* types,
                         const double* cell, const double* masses, double dt, int n_steps, double gamma_select,
                         double gamma_break, int ring_capacity, double* ring_pos, int32_t* ring_steps,
                         double* ring_gamma, int* n_selected, int* stop_step, double* gammas, double* e_pot,
                         double* e_kin, int* n_rebuilds, int flags, void* stream);

/*
 * Batched relaxation (the relaxation of candidate structures, Sec. 5: energy minimisation over atomic
 * positions and, with relax_cell = 1, the lattice vectors; each configuration ends relaxed or at
 * its first extrapolative configuration).  The paper names no minimiser; this is FIRE (Bitzek et
 * al. 2006: semi-implicit Euler, unit masses, N_min 5, f_inc 1.1, f_dec 0.5, a_start 0.1, f_a 0.99,
 * starting step dt, largest dt_max) on the coordinates q = [u, D]: H = H0 D^T, x = u D^T with D the
 * deformation gradient of the starting cell, forces F D on u and W D^-T / N on D (W the virial).
 * A configuration is converged when max |F| <= fmax and (relaxing the cell) max |W| / volume <=
 * smax; it stops when its grade (Sec. 2.3, the installed active set) reaches gamma_break (pass
 * INFINITY for no grade checks); every configuration, the starting one included, is checked.
 * Batch layout of mtp_eval_batch, device arrays; pos and cells are overwritten with the final
 * coordinates; energy [n_cfg] (device, the energy at the final coordinates), steps and status
 * ([n_cfg], host: 1 converged, 2 stopped by the grade, 3 step limit max_steps, 4 diverged) may be
 * NULL.  Synchronous.
 */
mtp_status mtp_relax_batch(mtp_model* model, int n_cfg, int n_atoms, const int32_t* cfg_off, double* pos,
                           const int32_t* types, double* cells, int relax_cell, double fmax, double smax,
                           double gamma_break, int max_steps, double dt, double dt_max, double* energy, int32_t* steps,
                           int32_t* status, void* stream);

/*
 * Training (Sec. 2.2: theta = (xi, c) minimises the loss of Eqs. 7, 11, 12; the paper names no
 * optimiser): limited-memory BFGS from the model's current parameters, with the last `history`
 * (s, y) pairs (two-loop recursion, H0 = s.y / y.y of the newest pair, before the first pair
 * I / max(1, max |g|); a pair with s.y <= 1e-12 |s| |y| is not kept) and a backtracking line search
 * (step 1 halved until L(theta + t d) <= L + 1e-4 t g.d, at most 40 halvings).  Every loss and
 * gradient is mtp_param_grad() on the batch (layout and arguments as there, device arrays);
 * direction, history and parameters stay on the device.  Stops when max |dL/dtheta| <= gtol
 * (status 0), after max_iter iterations (1) or when the line search fails (2).  The model keeps the
 * last accepted parameters.  losses ([max_iter + 1], host, L at each iterate), iterations and
 * status (host) may be NULL.  Synchronous.
 */
mtp_status mtp_train(mtp_model* model, int n_cfg, int n_atoms, const int32_t* cfg_off, const double* pos,
                     const int32_t* types, const double* cells, const double* e_ref, const double* f_ref,
                     const double* w_ref, double w_e, double w_f, double w_s, int scaling, int history, int max_iter,
                     double gtol, double* losses, int* iterations, int* status, void* stream);

/* Wait for the model's work on `stream` and report errors detected on the device since the last
 * check (MTP_EOVERFLOW, MTP_EINVAL for bad species or shifts). */
mtp_status mtp_sync(mtp_model* model, void* stream);

/* Number of kernel launches made by the model since creation (instrumentation). */
int64_t mtp_launch_count(const mtp_model* model);

/* Per-phase device timing (instrumentation).  While enabled, every synchronous evaluation records
 * CUDA events on its stream around the neighbour build and the four evaluation kernels (moments,
 * contraction, pair gradients, force/virial gather) and accumulates their elapsed times.
 * mtp_profile() resets the accumulators; mtp_profile_read() writes up to n totals in
 * milliseconds, in that order, and the number of evaluations accumulated. */
mtp_status mtp_profile(mtp_model* model, int enable);
mtp_status mtp_profile_read(const mtp_model* model, double* ms, int n, int64_t* calls);

/* Measured FP32 fused-multiply-add throughput of the current device in TFLOP/s (median of `repeats`
 * timed launches of a kernel of independent FMA chains that fills every SM; instrumentation for the
 * roofline of the float kernels, no counterpart in the paper).  Synchronous; allocates 4 bytes. */
mtp_status mtp_fp32_peak(int repeats, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* MTP_H */
