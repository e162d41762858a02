/*
 * nolsm.h — C ABI of the NOLSM density step on one GPU (libnolsm.so).
 *
 * The non-orthogonal local submatrix method (arXiv 2205.12182, Section II,
 * "Overview of the Problem"): for every column block C_b of the sparse,
 * non-orthogonal one-particle Hamiltonian H0 and overlap S, gather the dense
 * submatrices T_b(H0), T_b(S) on the rows where the combined pattern of the
 * block's columns is non-zero (step 1), evaluate
 *     T_b(D) = 1/2 (I - sign(T_b(S)^-1 T_b(H0) - mu I)) T_b(S)^-1      (Eq. 8)
 * with a Newton-Schulz-type sign iteration (Eq. 6) (step 2), and write the
 * block's own columns back into a sparse D with the input's pattern (step 3).
 * The chemical potential mu is set so that Tr(D S) equals the electron count
 * (Section V-A), and the band energy is Tr(D H0) (Eq. 4).
 *
 * Conventions for every call:
 *  - Functions return nolsm_status; no C++ exception crosses the ABI.  After an
 *    error the context is sticky-failed (every later call returns the same code)
 *    until nolsm_build_submatrices succeeds again; nolsm_last_error() says why.
 *  - Work is ordered on the CUDA stream given to nolsm_create.  Calls that return
 *    host scalars (nolsm_set_mu, nolsm_band_energy, nolsm_sign_batch statistics)
 *    synchronise that stream; the others only enqueue.
 *  - The caller owns every buffer it passes.  Device-resident H0/S values must
 *    stay valid and unchanged until the next nolsm_build_submatrices or
 *    nolsm_destroy (the context reads them again for the band energy); host-
 *    resident inputs are copied.  The context owns its submatrix, factor,
 *    iterate and scratch buffers and frees them in nolsm_destroy.
 *  - Matrices are square, symmetric, and H0 and S share one CSR pattern:
 *    int64 row pointers, int32 column indices ascending within each row,
 *    float64 values.  The pattern must be structurally symmetric and hold the
 *    full diagonal.
 */
#ifndef NOLSM_H
#define NOLSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NOLSM_ABI_VERSION 1

typedef enum nolsm_status {
  NOLSM_OK = 0,
  NOLSM_EINVAL = 1,      /* bad argument, size or pattern */
  NOLSM_ENOMEM = 2,      /* device or host allocation failed */
  NOLSM_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  NOLSM_ENOTPD = 4,      /* a submatrix T_b(S) is not positive definite */
  NOLSM_ENOCONV = 5,     /* ||X^2 - I||_F above tolerance after max_iter */
  NOLSM_EBRACKET = 6,    /* N(mu) does not bracket the electron count */
  NOLSM_ETIMEOUT = 7,    /* a bounded device-side wait ran out */
  NOLSM_ENOTBUILT = 8,   /* call needs nolsm_build_submatrices / nolsm_sign_batch first */
  NOLSM_ENONFINITE = 9   /* NaN or Inf met in the inputs or an iterate */
} nolsm_status;

typedef enum nolsm_memory {
  NOLSM_MEM_DEVICE = 0,  /* pointer is device memory of the context's GPU */
  NOLSM_MEM_HOST = 1     /* pointer is host memory (pinned or pageable) */
} nolsm_memory;

typedef enum nolsm_precision {
  /* Sign iteration with FP32 operands and FP32 accumulation (SIMT). */
  NOLSM_PREC_FP32 = 1,
  /* FP16 operands, FP32 accumulation on the tensor cores (tcgen05, TMEM);
   * the own-column slab gets the final Newton-Schulz steps in FP32. */
  NOLSM_PREC_MIXED_FP16 = 2,
  /* As MIXED_FP16 with BF16 operands (an accuracy/throughput variant). */
  NOLSM_PREC_MIXED_BF16 = 3
} nolsm_precision;

typedef enum nolsm_bounds {
  NOLSM_BOUNDS_GERSHGORIN = 0,  /* Gershgorin discs of A0 = L^-1 T(H0) L^-T */
  NOLSM_BOUNDS_LANCZOS = 1,     /* Lanczos extreme Ritz values of A0 widened by the last Lanczos
                                   coefficient; the first iteration is unscaled (see nolsm_sign_batch) */
  NOLSM_BOUNDS_LEARNED = 2,     /* network predictions (nolsm_set_predictor) for the scale and the lower
                                   bound; capped by Gershgorin, first iteration unscaled, a block whose
                                   residual blows up restarts from the Gershgorin scale */
  NOLSM_BOUNDS_GIVEN = 3        /* per-block (lambda_min, lambda_max, log10 distance of mu to the
                                   spectrum) kept from an earlier geometry with the same blocks
                                   (nolsm_keep_bounds: the next MD or SCF step) or set by the caller
                                   (nolsm_set_block_bounds), used as the network's predictions are
                                   (same caps, floors and restart); Gershgorin while none are held */
} nolsm_bounds;

typedef enum nolsm_chol_precision {
  NOLSM_CHOL_FP64 = 0,          /* Cholesky factor of T_b(S) in FP64, its triangular inverse in FP32 */
  NOLSM_CHOL_FP32 = 1,          /* factor and inverse in FP32 */
  NOLSM_CHOL_FP64_INV64 = 2,    /* factor and inverse in FP64 */
  NOLSM_CHOL_DF64 = 3,          /* factor in double-float pairs (Dekker; 48-bit significand), stored as
                                   FP64; inverse in FP32.  Blocked by 64-column panels: each panel's
                                   64x64 diagonal block in double-float on the FP32 pipe, the rows
                                   below it and the trailing updates on the tensor cores from exact
                                   8-bit slices (Ozaki scheme, 48 bits).  The factor feeds the rest of the path through its FP32
                                   rounding (and the trace slab), where it agrees with the FP64 factor */
  NOLSM_CHOL_DF64_SIMT = 4      /* the same double-float factor with every update on the FP32 pipe
                                   (one left-looking launch) */
} nolsm_chol_precision;

/* How the tensor-core products of the mixed-precision paths are scheduled (the FP32 path always
 * launches one grouped product at a time). */
typedef enum nolsm_schedule {
  NOLSM_SCHEDULE_PERSISTENT = 0,  /* one launch per sign evaluation: 2-CTA clusters take whole blocks
                                     off a queue and run all of a block's products with its iterates
                                     resident in L2; convergence is decided on the device */
  NOLSM_SCHEDULE_PER_PRODUCT = 1, /* one grouped launch per product over all active blocks, the
                                     iteration driven from the host; from n_pad 1024 on, the tiles
                                     are dealt round-robin so that all SMs share a few blocks'
                                     operands in L2 */
  NOLSM_SCHEDULE_AUTO = 2,        /* the measured table of nolsm_set_schedule_table when one is set;
                                     otherwise PERSISTENT while every block has n_pad < 1024 (the
                                     iterates of the blocks in flight stay in L2), PER_PRODUCT otherwise */
  NOLSM_SCHEDULE_PERSISTENT_INTERLEAVED = 3  /* PERSISTENT with two blocks per cluster: the products
                                     of both alternate and share one cluster barrier per pair (same
                                     arithmetic).  Twice the iterates in flight: at n_pad 512 they no
                                     longer fit in L2, and it is slower than PERSISTENT there */
} nolsm_schedule;

/* Where the refinement steps on the own-column slab run on the mixed-precision paths (the FP32 path
 * always uses the SIMT kernels). */
typedef enum nolsm_refine_path {
  NOLSM_REFINE_TENSOR = 0,  /* tensor cores: X in its FP16/BF16 storage times the FP32 slab split into
                               two FP16/BF16 terms (hi + lo), FP32 accumulation; one persistent CTA per
                               block (and 192-column piece of its own columns) runs the whole chain */
  NOLSM_REFINE_SIMT = 1     /* FP32 SIMT products (blocks resident in an 8-CTA cluster's shared
                               memory, one CTA per block beyond that) */
} nolsm_refine_path;

/* First point of the chemical-potential bisection (nolsm_set_mu). */
typedef enum nolsm_mu_first {
  NOLSM_MU_FIRST_AUFBAU = 0,    /* the Aufbau estimate from the diagonal of A0, when inside the bracket */
  NOLSM_MU_FIRST_MIDPOINT = 1   /* the bracket midpoint: plain bisection from the first step */
} nolsm_mu_first;

/* How the per-product schedule drives its iteration (the persistent schedules run it inside their
 * one launch). */
typedef enum nolsm_loop {
  NOLSM_LOOP_GRAPH = 0,   /* one CUDA graph launch per sign evaluation: a conditional while node whose
                             body is one iteration (tile lists, both products, the convergence test)
                             and whose last kernel decides on the device whether another iteration runs;
                             the graph is captured once per build and reused at every mu */
  NOLSM_LOOP_HOST = 1     /* the same launches issued from the host, which polls the device flags every
                             fourth iteration */
} nolsm_loop;

/* One CSR matrix (see the conventions above). */
typedef struct nolsm_csr {
  int64_t n;               /* dimension N */
  int64_t nnz;             /* stored entries */
  const int64_t* row_ptr;  /* n+1 entries, row_ptr[0] = 0, row_ptr[n] = nnz */
  const int32_t* col;      /* nnz column indices, ascending within a row */
  const double* val;       /* nnz values */
  int32_t memory;          /* nolsm_memory of row_ptr, col and val */
} nolsm_csr;

typedef struct nolsm_options {
  int32_t precision;       /* nolsm_precision (default MIXED_FP16) */
  int32_t bounds;          /* nolsm_bounds (default GERSHGORIN) */
  int32_t chol_precision;  /* nolsm_chol_precision (default DF64) */
  int32_t scaled;          /* 1: scaled Newton-Schulz (Chen & Chow 2014), 0: Eq. 6 as written */
  double sign_tol;         /* stop the full-matrix iteration when ||X^2 - I||_F <= sign_tol; <= 0 picks
                              min(0.05, max(8 u sqrt(n_b), t)) with u the operand format's unit roundoff
                              and t = 0.02, 4e-4, 0 for refine_iters >= 2, 1, 0 (the refinement steps
                              on the own columns finish the convergence) */
  int32_t max_iter;        /* matrix iterations per sign evaluation (default 100) */
  int32_t refine_iters;    /* FP32 Newton-Schulz steps on the own-column slab (0..3, default 2) */
  double spin_factor;      /* electrons per orbital: N_e = spin_factor Tr(DS), E = spin_factor Tr(DH0) (default 2) */
  double lower_bound;      /* scaled iteration: lower bound on |eig(X_0)| when bounds give none (default 0.02;
                              a bound far below the truth costs FP16 accuracy, one above it iterations) */
  double alpha_margin;     /* relative safety margin on the spectral radius bound (default 0.02) */
  int64_t wait_budget;     /* bound on every device-side spin wait, in polls (default 1<<22) */
  int32_t lanczos_steps;   /* Lanczos steps per block for NOLSM_BOUNDS_LANCZOS (default 24, at most 64) */
  int32_t schedule;        /* nolsm_schedule of the mixed-precision products (default AUTO) */
  int32_t refine_path;     /* nolsm_refine_path of the mixed-precision paths (default TENSOR) */
  int32_t fp8_iters;       /* experiment (mixed paths, schedule PERSISTENT or AUTO resolving to it): the first fp8_iters
                              Newton-Schulz iterations round both product outputs (B and X+) to FP8 E4M3
                              values before storing them, i.e. FP8 operands without the FP8 MMA rate
                              (default 0, at most max_iter) */
  int32_t mu_first;        /* nolsm_mu_first of nolsm_set_mu (default AUFBAU) */
  int32_t loop;            /* nolsm_loop of the per-product schedule (default GRAPH) */
} nolsm_options;

/* Statistics of the last sign evaluation. */
typedef struct nolsm_sign_stats {
  double mu;               /* chemical potential of the evaluation */
  double n_electrons;      /* spin_factor * Tr(D S) over all blocks' own columns */
  double band_energy;      /* spin_factor * Tr(D H0) from the same block traces */
  double max_residual;     /* max over blocks of ||X^2 - I||_F at exit of the matrix iteration */
  double iters_avg;        /* matrix iterations (each = two matrix products) per block */
  int32_t iters_min;
  int32_t iters_max;
  int32_t n_blocks;
  int32_t n_restarted;     /* blocks restarted with the Gershgorin bound after residual growth */
  double flops_paper;      /* 2 n_b^3 per product, true n_b (the paper's count, Section V-B) */
  double flops_executed;   /* as executed: padded n, upper-triangular tiles (n_pad^2 (n_pad + 128) per product) */
  double ms;               /* device time of the evaluation (CUDA events) */
} nolsm_sign_stats;

typedef struct nolsm_ctx nolsm_ctx;

/* Fill *opt with the defaults listed above. */
nolsm_status nolsm_default_options(nolsm_options* opt);

/* Create a context on the current CUDA device; cuda_stream is a cudaStream_t (NULL =
 * legacy default stream).  opt may be NULL for defaults.  *ctx is set on success. */
nolsm_status nolsm_create(nolsm_ctx** ctx, const nolsm_options* opt, void* cuda_stream);

/* Step 1 of the submatrix method and everything that does not depend on mu
 * (Section II; Eq. 8).  For block b with own columns blk_cols[blk_ptr[b]..blk_ptr[b+1])
 * the index set I_b is every row holding a stored entry in one of those columns,
 * unioned with extra_idx[extra_ptr[b]..extra_ptr[b+1]) when extra_ptr is not NULL
 * (a geometric neighbourhood).  blk_* and extra_* are host arrays.  The call
 * gathers T_b(H0) and T_b(S), factors T_b(S) = L L^T, forms A0 = L^-1 T_b(H0) L^-T
 * (so that sign(T_b(S)^-1 T_b(H0) - mu) = L^-T sign(A0 - mu) L^T) and its spectral
 * bounds.  n_b = |I_b| must not exceed 16384 (Table II's submatrices reach 10,737); while every
 * block has n_b <= 4096 the index sets take 4096 entries per block, otherwise 16384.  Blocks with
 * n_pad > 4096 run the per-product schedule whatever nolsm_options.schedule says.  Errors: EINVAL
 * (sizes, pattern, n_b), ENOTPD, ENONFINITE, ENOMEM, ECUDA. */
nolsm_status nolsm_build_submatrices(nolsm_ctx* ctx, const nolsm_csr* H, const nolsm_csr* S,
                                     int32_t n_blocks, const int32_t* blk_ptr, const int32_t* blk_cols,
                                     const int32_t* extra_ptr, const int32_t* extra_idx);

/* Step 2 at one chemical potential (Eq. 8 with the iteration of Eq. 6): for every
 * block, X -> sign(A0 - mu I), then the block traces of D S and D H0 over its own
 * columns.  Fills *out when out is not NULL (synchronises).  Errors: ENOTBUILT,
 * ENOCONV, ETIMEOUT, ENONFINITE, ECUDA. */
nolsm_status nolsm_sign_batch(nolsm_ctx* ctx, double mu, nolsm_sign_stats* out);

/* Chemical potential by bisection (Section V-A: the mu that makes the system
 * charge neutral).  With nolsm_options.mu_first = AUFBAU (the default) the first point
 * is an Aufbau estimate when it lies inside the bracket (MIDPOINT: the bracket
 * midpoint, plain bisection): with k = floor(n_electrons / spin_factor) occupied orbitals, the midpoint
 * of the k-th and (k+1)-th smallest diagonal entries of A0 over the blocks' own
 * columns; every later step evaluates nolsm_sign_batch at the bracket midpoint.
 * It stops when |N(mu) - n_electrons| <= tol_n * n_electrons, when the bracket is
 * below 1e-10 Ha, or after max_steps.  mu_lo >= mu_hi selects the bracket
 * [min lower bound, max upper bound] over the blocks.  Outputs may be NULL.
 * Errors: EBRACKET (the bracket does not contain the count), plus those of
 * nolsm_sign_batch. */
nolsm_status nolsm_set_mu(nolsm_ctx* ctx, double n_electrons, double mu_lo, double mu_hi, double tol_n,
                          int32_t max_steps, double* mu_out, double* n_out, int32_t* steps_out);

/* Step 3 at the mu of the last sign evaluation: D_b[:, C_b] = L^-T 1/2 (I - X) L^-1[:, C_b]
 * written into d_val (nnz values on the H0/S pattern; entries (i, c) with c an
 * own column of exactly one block; entries of columns owned by no block are 0).
 * memory says where d_val lives; d_val may be NULL to keep D inside the context
 * only (nolsm_band_energy uses it).  Errors: ENOTBUILT, EINVAL, ECUDA. */
nolsm_status nolsm_density(nolsm_ctx* ctx, double* d_val, int32_t memory);

/* Band energy spin_factor * Tr(D H0) = spin_factor * sum_ij D_ij H0_ji (Eq. 4) of the D
 * assembled by the last nolsm_density, accumulated in FP64.  Synchronises. */
nolsm_status nolsm_band_energy(nolsm_ctx* ctx, double* e_out);

/* Result of nolsm_solve_chunked. */
typedef struct nolsm_chunked_stats {
  double mu;                 /* chemical potential of the last pass (D is the D at this mu) */
  double n_electrons;        /* spin_factor * Tr(D S) at mu, summed over every block */
  double band_energy;        /* spin_factor * Tr(D H0) of the assembled D (Eq. 4), FP64 */
  double band_energy_traces; /* the same from the blocks' traces (a cross-check) */
  double iters_avg;          /* matrix iterations per block in the last pass */
  double flops_paper;        /* products of the last pass, 2 n_b^3 each (the paper's count) */
  double flops_executed;     /* products of the last pass as executed (n_pad^2 (n_pad + 128) each) */
  double flops_useful;       /* products of the last pass, n_b^2 (n_b + 1) each (one triangle and the
                                diagonal of a symmetric product) */
  double ms_total;           /* device time of the call (CUDA events on the context stream) */
  double ms_last_pass;       /* device time of the last pass: every chunk built, evaluated, scattered */
  int32_t iters_max;
  int32_t passes;            /* sign evaluations of every block (one per chemical potential tried) */
  int32_t chunks;
  int32_t n_blocks;
  int32_t max_chunk_blocks;
  int32_t reserved;
} nolsm_chunked_stats;

/* The whole density step -- build, chemical potential, density, band energy -- for a system whose
 * blocks' dense matrices do not fit in device memory at once (the submatrix method's blocks are
 * independent, Section II).  The CSR of H0 and S (device memory, as for nolsm_build_submatrices) and
 * the caller's D stay resident; the blocks are streamed through the context's pools in chunks of
 * consecutive blocks.  Each pass builds every chunk in turn (nolsm_build_submatrices on the chunk),
 * evaluates its sign at the pass's mu (nolsm_sign_batch), adds its terms of N(mu) = Tr(D S) and
 * Tr(D H0), and scatters its columns of D into d_val.  mu follows nolsm_set_mu's bisection (Section
 * V-A) with one pass per evaluation: the first point is the Aufbau estimate of the first chunk (its
 * own columns with their share of the n_electrons / spin_factor occupied orbitals), the second the
 * Aufbau estimate over every block when it lies inside the bracket [min lower bound, max upper
 * bound] (known after the first pass), then midpoints; it stops when |N(mu) - n_electrons| <=
 * tol_n * n_electrons, when the bracket is below 1e-10 Ha, or after max_passes.
 *   chunk_blocks  blocks per chunk; <= 0 sizes the chunks from an estimate of their pools (index-set
 *                 bound from the own rows' entries and the extra list) within 60 % of the free
 *                 device memory.
 *   d_val         device, nnz float64, caller-owned: D on the H0/S pattern at the returned mu
 *                 (entries of columns owned by no block are 0).
 *   block_n, block_e  host arrays of n_blocks or NULL: every block's terms of N and E at the returned
 *                 mu (as nolsm_block_traces).
 *   out           may be NULL.
 * The context keeps the last chunk's build afterwards; nolsm_density and nolsm_band_energy refer to it
 * (call nolsm_build_submatrices before using the context otherwise).  Synchronises.  Errors: those
 * of nolsm_build_submatrices and nolsm_sign_batch, EINVAL (host-resident CSR, bad arguments),
 * EBRACKET. */
nolsm_status nolsm_solve_chunked(nolsm_ctx* ctx, const nolsm_csr* H, const nolsm_csr* S, int32_t n_blocks,
                                 const int32_t* blk_ptr, const int32_t* blk_cols, const int32_t* extra_ptr,
                                 const int32_t* extra_idx, int32_t chunk_blocks, double n_electrons, double tol_n,
                                 int32_t max_passes, double* d_val, double* block_n, double* block_e,
                                 nolsm_chunked_stats* out);

/* Measured schedule table for NOLSM_SCHEDULE_AUTO (the library's autotuner,
 * paper_2205_12182_gb300/autotune.py, writes one from timings of the products at each n_pad): entry i
 * says which schedule ran the products of blocks with n_pad[i-1] < n_pad <= n_pad[i] fastest (the
 * first entry covers everything below, the last everything above).  ms_per_block (NULL, or
 * 3 n_entries values: per entry the products' time per block and sign evaluation under PERSISTENT,
 * PER_PRODUCT and PERSISTENT_INTERLEAVED, measured in full batches) lets AUTO predict a batch:
 *  - without times, every sign evaluation takes the blocks whose entry is PERSISTENT or
 *    PERSISTENT_INTERLEAVED into one persistent launch (largest first; the variant preferred by the
 *    larger share of their n_pad^3) and runs the others, and every block above n_pad 4096, with
 *    per-product launches after it (a split evaluation);
 *  - with times, AUTO predicts the batch's products time under each single schedule (the sum of its
 *    blocks' times) and under that split (plus the persistent launch's tail: its last block alone,
 *    about its time per block times the clusters) and runs the smallest.
 * n_pad ascending and positive, schedule one of PERSISTENT, PER_PRODUCT, PERSISTENT_INTERLEAVED, times
 * positive; n_entries = 0 removes the table (AUTO is then persistent while every n_pad < 1024).
 * Copied.  Errors: EINVAL. */
nolsm_status nolsm_set_schedule_table(nolsm_ctx* ctx, int32_t n_entries, const int32_t* n_pad, const int32_t* schedule,
                                      const double* ms_per_block);

/* Schedule of the last sign evaluation: *schedule = PERSISTENT, PERSISTENT_INTERLEAVED or PER_PRODUCT
 * when every block ran it, -2 when the evaluation was split (a persistent launch, then per-product
 * launches); *persistent_blocks = blocks of the persistent launch.  Either may be NULL.
 * Errors: ENOTBUILT (no sign evaluation). */
nolsm_status nolsm_last_schedule(const nolsm_ctx* ctx, int32_t* schedule, int32_t* persistent_blocks);

/* Number of blocks, and n_b / |C_b| of block b (host query of the build). */
nolsm_status nolsm_block_info(const nolsm_ctx* ctx, int32_t b, int32_t* n_b, int32_t* n_cols);

/* Diagonal entries of A0 = L^-1 T_b(H0) L^-T at every block's own columns (the data of
 * nolsm_set_mu's Aufbau first point), in block order: *count = sum_b |C_b|, copied to out (host,
 * *count floats) when out is not NULL.  Lets ranks that hold different blocks agree on the same
 * first point.  Errors: EINVAL (not built, count NULL). */
nolsm_status nolsm_own_diagonal(const nolsm_ctx* ctx, int64_t* count, float* out);

/* Per-block terms of the last sign evaluation's electron count and band energy (host arrays of
 * n_blocks; either may be NULL): n_out[b] = spin_factor * sum_{j in C_b} (T_b(S) T_b(D))_jj and
 * e_out[b] = spin_factor * sum_{j in C_b} (T_b(H0) T_b(D))_jj, the block's share of Tr(D S) and
 * Tr(D H0) at that evaluation's mu (Eq. 4, Section V-A), accumulated in FP64.  Their sums are the
 * evaluation's n_electrons and band_energy.  Synchronises.  Errors: ENOTBUILT (no sign evaluation),
 * EINVAL (both outputs NULL), ECUDA. */
nolsm_status nolsm_block_traces(const nolsm_ctx* ctx, double* n_out, double* e_out);

/* Index set I_b of block b copied to idx_out (host, n_b entries). */
nolsm_status nolsm_block_index_set(const nolsm_ctx* ctx, int32_t b, int32_t* idx_out);

/* Per-block spectral bounds [lo, hi] of A0 used by the iteration (host arrays of n_blocks). */
nolsm_status nolsm_block_bounds(const nolsm_ctx* ctx, double* lo, double* hi);

/* Per-block state of the last sign evaluation (host arrays of n_blocks; any may be NULL):
 * completed matrix iterations, ||X^2 - I||_F of the last product, and the exit status
 * (0 still iterating, 1 converged, 2 restarted, 3 failed).  Synchronises. */
nolsm_status nolsm_block_state(const nolsm_ctx* ctx, int32_t* iters, double* residual, int32_t* status);

/* Diagnostic copy of block b's n_b x n_b matrix `which` to host memory (row-major, float32):
 * which = 0: A0 = L^-1 T_b(H0) L^-T;  1: L^-1;  2, 3: the two iterate buffers X;  4: the
 * second-operand buffer of the last product;  5: the Cholesky factor L of T_b(S) (FP32 rounding
 * of the factor as computed, zero above the diagonal).  Synchronises. */
nolsm_status nolsm_block_matrix(const nolsm_ctx* ctx, int32_t b, int32_t which, float* out);

/* Diagnostic copy of block b's Cholesky factor L of T_b(S) at the precision it was computed in
 * (FP64 modes: the FP64 lower triangle; double-float modes: each pair's value h + l; CHOL_FP32: the
 * FP32 factor widened), n_b x n_b row-major in host memory, zero above the diagonal.  Synchronises. */
nolsm_status nolsm_block_factor(const nolsm_ctx* ctx, int32_t b, double* out);

/* Cumulative counters of ctx since nolsm_create or the last reset (reset != 0 zeroes them after
 * reading): kernels launched by the library, and the device time (CUDA events on the context
 * stream, ms) and executed flops of the Newton-Schulz matrix-product launches.  Synchronises. */
nolsm_status nolsm_counters(nolsm_ctx* ctx, int64_t* launches, int64_t* gemm_launches, double* gemm_ms,
                            double* gemm_flops, int32_t reset);

/* Replace the poll budget of every device-side wait (nolsm_options.wait_budget) for the calls that
 * follow; budget >= 1.  A wait that runs out records NOLSM_ETIMEOUT (see nolsm_sign_batch). */
nolsm_status nolsm_set_wait_budget(nolsm_ctx* ctx, int64_t budget);

/* Stages of the path timed by nolsm_phase_times. */
typedef enum nolsm_phase {
  NOLSM_PHASE_GATHER = 0,      /* index sets done: dense T_b(H0), T_b(S) from the CSR rows (step 1) */
  NOLSM_PHASE_FACTOR = 1,      /* Cholesky factor of every T_b(S) (double-float blocked mode: the 64 x 64
                                  diagonal blocks and the FP32 copy; its other two parts below) */
  NOLSM_PHASE_INVERSE = 2,     /* triangular inverses L^-1 */
  NOLSM_PHASE_CONGRUENCE = 3,  /* A0 = L^-1 T_b(H0) L^-T */
  NOLSM_PHASE_BUILD_REST = 4,  /* own-column slabs, bounds, block features, tensor maps */
  NOLSM_PHASE_SIGN_SETUP = 5,  /* per evaluation: features at mu, predictions, initial scales */
  NOLSM_PHASE_PRODUCTS = 6,    /* the Newton-Schulz matrix products and their iteration control */
  NOLSM_PHASE_SLAB = 7,        /* own-column refinement and the block traces */
  NOLSM_PHASE_DENSITY = 8,     /* back-transform and scatter of D (step 3) */
  NOLSM_PHASE_ENERGY = 9,      /* Tr(D H0) */
  NOLSM_PHASE_FACTOR_TRSM = 10,    /* blocked double-float factor: rows below each diagonal block */
  NOLSM_PHASE_FACTOR_UPDATE = 11,  /* blocked double-float factor: tensor-core trailing updates */
  NOLSM_NUM_PHASES = 12
} nolsm_phase;

/* Cumulative device time of each nolsm_phase (ms, CUDA event pairs recorded on the context stream
 * around the stage's launches) since nolsm_create or the last reset: ms[p] for p < n (n at most
 * NOLSM_NUM_PHASES).  reset != 0 zeroes them after reading.  Synchronises. */
nolsm_status nolsm_phase_times(nolsm_ctx* ctx, double* ms, int32_t n, int32_t reset);

/* Band energy spin_factor * sum_e d_val[e] * h_val[e] over nnz stored entries (the reduction of
 * nolsm_band_energy), for callers that must not allocate device memory at the point of the call:
 * code between the steps of a molecular-dynamics integrator that runs under a fixed device-memory
 * budget, runtimes that route every device allocation through their own pool, or a hot loop where
 * an allocation would synchronise the device.  The call needs no context, makes no
 * cudaMalloc/cudaFree or other allocating call, and keeps its partial sums in a fixed 128 KB array
 * in device memory that the library declares at file scope.  d_val and h_val are device arrays on
 * one symmetric pattern (so H0_ji = H0_ij), e_out is one device double, all owned by the caller;
 * work is enqueued on cuda_stream (a cudaStream_t, NULL = legacy default stream) and the call
 * returns without synchronising.  The paper has no counterpart: this is a library convenience.
 * Limits and behaviour:
 *  - nnz may not exceed 268,435,456 (16,384 partial sums of 16,384 entries); larger inputs,
 *    nnz <= 0, null pointers or spin_factor <= 0 return NOLSM_EINVAL before any launch.
 *  - The array's code module is loaded into a context lazily (CUDA's default lazy loading): the
 *    first call on each device (each context) loads it, which allocates the array and the code
 *    and may synchronise.  A caller with a fixed memory budget makes one warm-up call before the
 *    budget applies; make that first call before any stream capture.  Every call looks up the
 *    array's device address (cudaGetSymbolAddress) in the current context, so a context created
 *    after a cudaDeviceReset gets its own array.
 *  - Every call in a context shares the array and leaves its partial sums in it; calls whose work
 *    overlaps on the GPU (other streams, no ordering between them) race on it.
 *  - A CUDA error left pending by earlier work is cleared (not reported) before the first launch;
 *    returns NOLSM_ECUDA when the lookup or one of this call's launches fails. */
nolsm_status nolsm_band_energy_noalloc(int64_t nnz, const double* d_val, const double* h_val, double spin_factor,
                                       double* e_out, void* cuda_stream);

/* ---- learned spectral bounds -------------------------------------------------------------
 * A network 32 -> 128 -> 128 -> 3 (GELU) predicts per block, from 32 features of A0 at a given mu,
 * lambda_min(A0), lambda_max(A0) and log10 of the distance from mu to the nearest eigenvalue of
 * A0.  The paper leaves the scaling of the sign iteration open (Section II, Eq. 6); these
 * predictions set the scale and the lower bound of the scaled iteration.  Parameters are one
 * float32 vector of 21,123 entries in the order W1 (128x32, row-major), b1, W2 (128x128), b2,
 * W3 (3x128), b3; `norm` is 70 floats: feature means (32), feature scales (32), target means (3),
 * target scales (3); inputs and targets are standardised with them inside the kernels. */

/* Features of every block at mu into feat (device, n_blocks x 32 float32, row per block):
 * n/512, |C_b|/n, mu, Gershgorin lo and hi, mean/std/min/max of diag(A0), ||offdiag||_F/sqrt(n),
 * mean/max/std of the Gershgorin radii, Tr(A0^2)/n, Tr(A0)/n, sqrt(Tr(A0^2)/n - (Tr A0/n)^2),
 * mean(diag) - mu, min|diag - mu|, fractions of diag below mu / within 0.05 / within 0.1 Ha of mu,
 * mean and max |offdiag|, skewness and kurtosis of diag, fraction of discs containing mu, min and
 * mean (|a_ii - mu| - R_i), relative position of mu in the Gershgorin interval, log10 of the
 * Gershgorin scale, |C_b|/100, 1.  Enqueued only. */
nolsm_status nolsm_block_features(nolsm_ctx* ctx, double mu, float* feat);

/* Lanczos on every block (steps <= 64, full reorthogonalisation): op 0 on A0, op 1 on
 * |A0 - mu| = X (A0 - mu) with X the iterate of the last nolsm_sign_batch (its mu).  out (device,
 * n_blocks x 4 float32): smallest and largest Ritz value, last Lanczos coefficient, steps taken.
 * Synchronises. */
nolsm_status nolsm_block_lanczos(nolsm_ctx* ctx, int32_t steps, int32_t op, float* out);

typedef struct nolsm_mlp nolsm_mlp;

/* Create a network on the current device (params: host, or NULL for zeros; norm: host, 70). */
nolsm_status nolsm_mlp_create(nolsm_mlp** mlp, const float* params, const float* norm, void* cuda_stream);
/* Copy the FP32 parameters to host memory (21,123 floats).  Synchronises. */
nolsm_status nolsm_mlp_get_params(const nolsm_mlp* mlp, float* params);
/* Gradient of (1/n) sum_s 1/2 sum_k w_k (y_k - t_k)^2 over n samples (x: device n x 32, t: device
 * n x 3, both raw; w: host 3 weights) with the FP32 parameters; kept for nolsm_mlp_adam and
 * copied to grad (device, 21,123) when not NULL; loss to *loss (host) when not NULL (synchronises). */
nolsm_status nolsm_mlp_gradient(nolsm_mlp* mlp, const float* x, const float* t, int32_t n, const float* w,
                                float* grad, double* loss);
/* One Adam step (bias-corrected moments) with the last gradient; refreshes the BF16 copy. */
nolsm_status nolsm_mlp_adam(nolsm_mlp* mlp, float lr, float beta1, float beta2, float eps);
/* Predictions for n samples (x: device n x 32 raw features; y: device n x 3) with BF16 weights and
 * FP32 accumulation. */
nolsm_status nolsm_mlp_predict(const nolsm_mlp* mlp, const float* x, int32_t n, float* y);
void nolsm_mlp_destroy(nolsm_mlp* mlp);

/* Bounds for the next geometry (the paper reruns the density step every MD time step, Section I;
 * one geometry's spectra are a close guess for the next): Lanczos (steps <= 64, full
 * reorthogonalisation) on A0 of the current build and on |A0 - mu| = X (A0 - mu) with the last sign
 * evaluation's X and mu; keeps per block (smallest and largest Ritz value of A0, log10 of the
 * smallest Ritz value of |A0 - mu|) in the context, where they survive the next
 * nolsm_build_submatrices and serve NOLSM_BOUNDS_GIVEN while that build has as many blocks.
 * Synchronises.  Errors: EINVAL (not built, steps out of range), ENOTBUILT (no sign evaluation
 * yet), ENOMEM, ECUDA. */
nolsm_status nolsm_keep_bounds(nolsm_ctx* ctx, int32_t steps);

/* Set the NOLSM_BOUNDS_GIVEN bounds directly: n_blocks x 3 float32 (lambda_min, lambda_max, log10
 * distance of mu to the spectrum) per block of the current build, in host or device memory
 * (nolsm_memory), copied.  Synchronises.  Errors: EINVAL (not built, null), ENOMEM, ECUDA. */
nolsm_status nolsm_set_block_bounds(nolsm_ctx* ctx, const float* bounds, int32_t memory);

/* Use mlp (kept by the caller, alive while ctx uses it) for NOLSM_BOUNDS_LEARNED; NULL detaches. */
nolsm_status nolsm_set_predictor(nolsm_ctx* ctx, const nolsm_mlp* mlp);

/* ---- submatrix combination ---------------------------------------------------------------
 * Section III-B-1: column blocks whose submatrices overlap strongly are cheaper solved as one.
 * Combining blocks a and b gives one block with own columns C_a u C_b and index set I_a u I_b, of
 * dimension n_a + n_b - n_ab (n_ab = |I_a n I_b|).  It pays iff t(n_a + n_b - n_ab) < t(n_a) + t(n_b)
 * with t(n) = n^3 (Eq. 9) or t(n) = p(n) n^3 (Eq. 10), p(n) the measured time per flop of the
 * matrix products at dimension n. */
typedef enum nolsm_combine_criterion {
  NOLSM_COMBINE_CUBIC = 0,        /* Eq. 9: flops of the dense products */
  NOLSM_COMBINE_PERFORMANCE = 1   /* Eq. 10: predicted run time p(n) n^3 */
} nolsm_combine_criterion;

/* Combine the column blocks of nolsm_build_submatrices' arguments (host work only: no context, no
 * GPU, thread safe).  Index sets follow nolsm_build_submatrices (the own columns' rows in the
 * pattern, the own columns, the extra list).  Order (the paper leaves it to earlier work): blocks
 * are candidates when the index set of one holds an own column of the other; each step combines the
 * candidate pair with the largest saving t(n_a) + t(n_b) - t(n_merged) > 0 whose merged dimension is
 * at most max_dim (ties: smallest pair of ids), the combined block keeps the smaller id, and the
 * loop stops when no candidate pays.
 *   pattern        host CSR (row_ptr, col; val unused) of H0 and S, structurally symmetric.
 *   blk_*, extra_* as for nolsm_build_submatrices; every column is owned by at most one block.
 *   criterion      nolsm_combine_criterion.
 *   pn_dim, pn_time (NOLSM_COMBINE_PERFORMANCE only; n_points >= 1 entries): sizes, strictly
 *                  ascending and >= 1, and the measured time per flop at each (positive, finite);
 *                  p(n) is linear in n between neighbouring sizes and constant beyond the ends.
 *   max_dim        largest dimension a combination may produce (input blocks above it stay alone).
 * Outputs (caller-owned host arrays; all but n_out and group may be NULL):
 *   *n_out         number of combined blocks m, numbered in ascending order of their smallest
 *                  input block;
 *   group          n_blocks entries: the combined block of each input block;
 *   out_blk_ptr    m + 1 entries (room for n_blocks + 1) and out_blk_cols (room for
 *                  blk_ptr[n_blocks]): each combined block's own columns, its input blocks' columns
 *                  in ascending block order;
 *   out_extra_ptr  m + 1 entries (room for n_blocks + 1) and out_extra_idx (room for
 *                  extra_ptr[n_blocks]): the sorted distinct union of the members' extra lists
 *                  (only with extra input);
 *   out_dim        m entries (room for n_blocks): n of each combined block;
 *   cost           2 doubles: the sum of t(n) over the input blocks and over the combined blocks.
 * Errors: EINVAL (null or inconsistent arguments, device memory, an index out of range, a column
 * owned twice, a bad p table, max_dim < 1), ENOMEM.  Nothing is written on error. */
nolsm_status nolsm_combine_blocks(const nolsm_csr* pattern, int32_t n_blocks, const int32_t* blk_ptr,
                                  const int32_t* blk_cols, const int32_t* extra_ptr, const int32_t* extra_idx,
                                  int32_t criterion, int32_t n_points, const int32_t* pn_dim, const double* pn_time,
                                  int32_t max_dim, int32_t* n_out, int32_t* group, int32_t* out_blk_ptr,
                                  int32_t* out_blk_cols, int32_t* out_extra_ptr, int32_t* out_extra_idx,
                                  int32_t* out_dim, double* cost);

/* Message of the last error of ctx (never NULL; "" when none).  ctx may be NULL. */
const char* nolsm_last_error(const nolsm_ctx* ctx);

/* Release every resource of ctx (NULL is a no-op). */
void nolsm_destroy(nolsm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* NOLSM_H */
