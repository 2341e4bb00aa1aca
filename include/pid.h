/*
 * pid.h — C ABI of the Probabilistic Inclusion Depth (PID) library for GB300 (sm_103a).
 *
 * The library computes, on one GPU, the data depth of every member of an ensemble of
 * N probabilistic (soft) masks u_i : {cells} -> [0,1] defined on M grid cells with
 * positive cell measures w_x (Sec. 3.2, Sec. 3.4 of the paper):
 *
 *   mass                m_i        = sum_x w_x u_i(x)                          (Eq. 6, Eq. 13)
 *   inclusion operator  u subset_p v = sum_x w u v / sum_x w u, 0 if m(u) = 0  (Eq. 9, Eq. 13)
 *   full PID            IN_in(i)  = (1/N) sum_j u_i subset_p u_j
 *                       IN_out(i) = (1/N) sum_j u_j subset_p u_i
 *                       PID(i)    = min(IN_in(i), IN_out(i))                   (Eq. 10, Eq. 14)
 *   PID-mean            u_bar = (1/N) sum_i u_i;  IN_in = u_i subset_p u_bar,
 *                       IN_out = u_bar subset_p u_i, depth = min              (Eq. 15, Eq. 16)
 *
 * and the fuzzy isocontour map of Sec. 3.5 that turns a scalar field F_i and an
 * isovalue distribution q ~ Normal(mu, sigma) into the soft mask
 *   u_i(x) = P(F_i(x) < q) = Phi((mu - F_i(x)) / sigma)        (inside = sub-level set, Eq. 2)
 * (sigma = 0 gives the indicator 1[F < mu]; `superlevel` selects P(F > q) instead).
 *
 * Conventions shared by every call
 *   - All array arguments are DEVICE pointers owned by the caller (for example the data
 *     pointers of torch CUDA tensors), except where a name ends in `_host`.
 *   - Ensemble data are row-major [N][ld] float32: member i, cell x at data[i*ld + x];
 *     ld >= M. Cell measures w are float32 [M], or NULL for unit measure (uniform grid,
 *     Eq. 12). Cell measures must be > 0 (Sec. 3.4). Rows that start on 16-byte
 *     boundaries (data and w 16-byte aligned, ld a multiple of 4) are staged by the tensor
 *     memory accelerator; other rows are read with plain loads, about 2.5x slower for the
 *     streaming passes, so pad ld to a multiple of 4 where the data allow it.
 *   - Outputs are float64 [N] (depths and inclusion fractions), int32 [N] (ranks:
 *     0 = deepest; ties go to the lower member index), float64 [N*N] (row-major inclusion
 *     matrix P[i*N + j] = u_i subset_p u_j). Any output pointer may be NULL to skip it.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL = legacy
 *     default stream). Outputs are valid once the stream has been synchronised.
 *   - Errors are returned, never raised with abort or a device trap. Argument errors are
 *     detected on the host before anything is enqueued. Errors found on the device (input
 *     out of [0,1] when validation is on, a bounded device wait that ran out) set a
 *     device-side error word of the handle; pid_sync() reports and clears it.
 *   - A handle owns device workspace. Calls made with one handle must not run
 *     concurrently on different streams; use one handle per concurrent stream.
 */
#ifndef PID_H_
#define PID_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pid_status {
  PID_OK = 0,
  PID_ERR_INVALID_ARG = 1,  /* bad size, stride, pointer or option (host-side check) */
  PID_ERR_DOMAIN = 2,       /* validation found u outside [0,1], a NaN, or w <= 0 */
  PID_ERR_OOM = 3,          /* workspace would exceed the handle's HBM budget, or cudaMalloc failed */
  PID_ERR_CUDA = 4,         /* a CUDA runtime call failed (see pid_last_error) */
  PID_ERR_TIMEOUT = 5,      /* a bounded device wait ran out; the kernel returned early */
  PID_ERR_BUSY = 6,         /* serving: queue full or server not accepting */
  PID_ERR_CANCELLED = 7,    /* serving: request cancelled or server stopped */
  PID_ERR_UNSUPPORTED = 8   /* size or option outside what this build implements */
} pid_status;

/* Which depth is computed. */
typedef enum pid_mode {
  PID_MODE_MEAN = 0,        /* PID-mean, Eq. 16: one streaming pass, O(NM) */
  PID_MODE_FULL = 1,        /* full PID, Eq. 10: N x N Gram G = U diag(w) U^T on tensor cores */
  PID_MODE_FULL_LINEAR = 2  /* full PID, exactly, in O(NM) (two streaming passes, FP32) */
} pid_mode;

/* Operand precision of the tensor-core Gram (PID_MODE_FULL). Accumulation is FP32, the
 * final normalisation FP64. PID_FP32 is accepted for FULL and selects FULL_LINEAR. */
typedef enum pid_precision {
  PID_FP32 = 0,
  PID_BF16 = 1,             /* u sqrt(w) rounded to bfloat16 */
  PID_SPLIT_BF16 = 2,       /* hi + lo bfloat16 pair; products hi*hi + hi*lo + lo*hi */
  PID_FP8 = 3               /* E4M3 with a power-of-two scale per member (see below) */
} pid_precision;

/*
 * E4M3 operands (PID_FP8). Member i's operands are u_i sqrt(w) s_i, with s_i the largest
 * power of two such that max_x u_i(x) sqrt(w_x) s_i <= 448, the largest finite E4M3 value;
 * the tensor-core Gram is unscaled exactly, G_ij = G'_ij / (s_i s_j), as it leaves tensor
 * memory. Because u subset_p v is unchanged by scaling u (Eq. 9), every member keeps E4M3's
 * 3-bit relative precision however small its values are. The scales take one extra read of
 * the ensemble (PID_KERNEL_SCALE) before the Gram. E4M3 rounding (up to 2^-4 of a value per
 * element) averages over cells: depths and IN_out stay within 1e-3 of the exact values from
 * 4096 cells on, but one inclusion P_ij is not averaged over members. So a PID_FP8 request
 * with fewer than 4096 cells (per time step, times the steps of a space-time ensemble) or
 * with P requested computes its Gram from BF16 operands instead; pid_gram_operands tells
 * which operands a request uses.
 */
pid_status pid_gram_operands(int32_t precision, int64_t cells, int32_t want_matrix,
                             int32_t* operands);

typedef enum pid_iso_kind {
  PID_ISO_NORMAL = 0,       /* isovalue q ~ Normal(mu, sigma), Sec. 3.5 */
  PID_ISO_UNIFORM = 1,      /* isovalue q ~ Uniform[mu - sigma, mu + sigma] (sigma > 0):
                               u = P(F < q) = clamp((mu + sigma - F) / (2 sigma), 0, 1) */
  PID_ISO_LEVEL = 2         /* level-centred map of the weather example (Sec. 3.6): probability
                               1 at the level mu, falling linearly to 0 at distance sigma:
                               u = max(0, 1 - |F - mu| / sigma) (sigma > 0, superlevel 0) */
} pid_iso_kind;

/* Isovalue distribution for pid_soft_masks / pid_from_fields (Sec. 3.5). */
typedef struct pid_iso {
  int32_t kind;             /* pid_iso_kind */
  int32_t superlevel;       /* 0: inside = {F < q} (Eq. 2); 1: inside = {F > q} */
  double mu;                /* mean isovalue */
  double sigma;             /* NORMAL: standard deviation, >= 0 (0 = hard threshold at mu);
                               UNIFORM, LEVEL: half-width, > 0 */
} pid_iso;

typedef struct pid_options {
  int32_t mode;             /* pid_mode */
  int32_t precision;        /* pid_precision (PID_MODE_FULL only) */
  int32_t validate;         /* 1: check u in [0,1] / finite fields and w > 0 on the device */
  int32_t reserved;         /* must be 0 */
} pid_options;

typedef struct pid_handle_s* pid_handle;

/* Create a handle on CUDA device `device`. `hbm_budget_bytes` caps the workspace the
 * handle may allocate (0 = no cap). Allocation happens lazily, on the first call that
 * needs more workspace (never while the stream is being captured). */
pid_status pid_create(pid_handle* out, int device, size_t hbm_budget_bytes);
/* Release the handle and its workspace. NULL is accepted. */
pid_status pid_destroy(pid_handle h);
/* Synchronise `stream`, then report (and clear) the handle's device error word. */
pid_status pid_sync(pid_handle h, void* stream);
/* Static text for a status code. */
const char* pid_status_string(pid_status s);
/* Detail text of the handle's most recent error (thread-unsafe; valid until the next call). */
const char* pid_last_error(pid_handle h);
/* Workspace bytes currently held by the handle. */
size_t pid_workspace_bytes(pid_handle h);

/*
 * Kernel timing. While enabled, the handle brackets each of its kernel launches with CUDA
 * events recorded on the launch stream and keeps, per kernel kind, the launch count, the
 * summed device time, and the algorithmic bytes and flops of those launches (bytes: one
 * read of every input element and cell measure, plus stored outputs; flops: 2 N^2 M per
 * Gram launch, times 3 for split BF16). Enabling resets the counters. Reading waits for
 * the recorded events.
 */
typedef enum pid_kernel_kind {
  PID_KERNEL_STREAM = 0,    /* PID-mean / exact full-PID streaming pass */
  PID_KERNEL_GRAM = 1,      /* tensor-core Gram, BF16 operands */
  PID_KERNEL_FINALIZE = 2,  /* FP64 reduction, depths, ranks */
  PID_KERNEL_ISO = 3,       /* isovalue map alone */
  PID_KERNEL_BANDS = 4,     /* contour boxplot bands */
  PID_KERNEL_GRAM_SPLIT = 5,  /* tensor-core Gram, split BF16 operands */
  PID_KERNEL_GRAM_FP8 = 6,  /* tensor-core Gram, E4M3 operands */
  PID_KERNEL_OPERANDS = 7,  /* operand staging of the row-block-tiled Gram (N > 256) */
  PID_KERNEL_SCALE = 8,     /* per-member E4M3 operand scales (one read of the ensemble) */
  PID_KERNEL_KINDS = 9
} pid_kernel_kind;

typedef struct pid_kernel_stats {
  int64_t launches;
  double total_ms;
  double bytes;
  double flops;
} pid_kernel_stats;

pid_status pid_profile_enable(pid_handle h, int enable);
pid_status pid_profile_read(pid_handle h, int kind, pid_kernel_stats* out);

/*
 * Autotuning. While enabled, the first launch of each kernel class and size bucket runs
 * every candidate of the launch parameters that leave results unchanged (the column-sum
 * exchange scheme and the TMA ring depth of the streaming kernel), times them with CUDA
 * events, and keeps the fastest for later launches. That first call synchronises its
 * stream; launches being captured into a CUDA graph are never tuned. If the environment
 * variable PID_AUTOTUNE_CACHE names a file, choices are loaded from it at pid_create and
 * appended to it as they are made. Returns the number of tuned entries in *n_entries
 * (may be NULL).
 */
pid_status pid_autotune_enable(pid_handle h, int enable, int32_t* n_entries);


/*
 * pid_soft_masks — the isovalue map alone (Sec. 3.5): U_out[i*ld_out + x] = u_i(x) for
 * x < M. F: [N][ld] float32 scalar fields; U_out: [N][ld_out] float32, ld_out >= M.
 * Cells x in [M, ld_out) of U_out are not written.
 */
pid_status pid_soft_masks(pid_handle h, const float* F, int64_t N, int64_t M, int64_t ld,
                          const pid_iso* iso, float* U_out, int64_t ld_out, void* stream);
/* The same map with bfloat16 output: U_out holds the bit patterns of the float32 masks
 * rounded to nearest even (2 bytes per element; the map itself runs in float32). */
pid_status pid_soft_masks_bf16(pid_handle h, const float* F, int64_t N, int64_t M, int64_t ld,
                               const pid_iso* iso, uint16_t* U_out, int64_t ld_out, void* stream);

/*
 * pid_selftest_wait_timeout — diagnostic of the bounded device waits, which every kernel
 * uses instead of unbounded spins (the paper has no counterpart). One thread waits on a
 * shared-memory mbarrier that nothing arrives at; after `seconds` (0 < seconds <= 2) the
 * bounded wait gives up and the kernel sets the timeout bit of the handle's device error
 * word, exactly as a stalled pipeline would. The next pid_sync returns PID_ERR_TIMEOUT and
 * clears the word; the context stays usable (nothing faults or traps).
 */
pid_status pid_selftest_wait_timeout(pid_handle h, double seconds, void* stream);

/*
 * pid_contour_bands — the bands of a contour boxplot (Sec. 6) from depths already
 * computed. Every member is binarised, b_i(x) = [u_i(x) > tau], with u_i the soft mask
 * itself (iso == NULL) or the isovalue map of the field (Sec. 3.5). For each cell x, the
 * byte bands[x] collects:
 *   bit 0 (1)   union of b_i over the inner population: the members whose rank is below
 *               ceil(inner_fraction * N) (rank 0 = deepest, as the depth calls return it)
 *   bit 1 (2)   intersection over the inner population
 *   bit 2 (4)   union over all members        bit 3 (8)  intersection over all members
 *   bit 4 (16)  b of the median member (rank 0)
 * The band of a population is union AND NOT intersection. data: [N][ld] float32 (any N);
 * rank: device int32 [N]; bands: device uint8 [M]. Requires 0 < tau < 1 and
 * 0 < inner_fraction <= 1 (PID_ERR_INVALID_ARG otherwise). The binarisation is decided
 * exactly: a field value is compared with the float nearest to the exact threshold F_tau
 * (u(F_tau) = tau) on the correct side, so no rounding of u enters the decision.
 */
pid_status pid_contour_bands(pid_handle h, const float* data, int64_t N, int64_t M, int64_t ld,
                             const pid_iso* iso, const int32_t* rank, double tau,
                             double inner_fraction, uint8_t* bands, void* stream);

/*
 * pid_mean — PID-mean (Eq. 15-16) of soft masks U [N][ld] with cell measures w [M] (or NULL).
 * Every member is compared with the mean contour u_bar; one fused pass over U.
 */
pid_status pid_mean(pid_handle h, const float* U, int64_t N, int64_t M, int64_t ld,
                    const float* w, double* depth, double* in_in, double* in_out,
                    int32_t* rank, void* stream);

/*
 * pid_full — full PID over all N^2 ordered pairs (Eq. 10 with the weighted sums of Eq. 14).
 * opt->mode = PID_MODE_FULL uses the tensor-core Gram in opt->precision and can return
 * the inclusion matrix P (N*N, row-major, P[i*N+j] = u_i subset_p u_j) and err_est[0],
 * the largest |IN_in(Gram) - IN_in(exact FP32)| over members, where the exact value comes
 * from the identity IN_in(i) = u_i subset_p u_bar (Eq. 17). opt->mode =
 * PID_MODE_FULL_LINEAR computes the same depths exactly in O(NM); P and err_est are then
 * not written. opt may be NULL (FULL_LINEAR, no validation).
 * The Gram modes take N <= 512 (PID_ERR_UNSUPPORTED above; FULL_LINEAR takes any N). Up to
 * 256 members one fused pass converts the operands on chip; from 257 to 512 the operand
 * rows are first staged in the handle's workspace (N * round_up(M, 64) * 2 bytes for BF16,
 * twice that for split BF16, half for E4M3) and the Gram runs over 128-row blocks.
 */
pid_status pid_full(pid_handle h, const float* U, int64_t N, int64_t M, int64_t ld,
                    const float* w, const pid_options* opt, double* depth, double* in_in,
                    double* in_out, int32_t* rank, double* P, double* err_est, void* stream);

/*
 * pid_from_fields — the isovalue map fused in front of the depth computation: u_i is
 * computed on the fly from the scalar fields F [N][ld] and `iso`, never stored. opt
 * selects PID-mean, full PID (Gram) or full PID (linear) exactly as for pid_mean/pid_full.
 */
pid_status pid_from_fields(pid_handle h, const float* F, int64_t N, int64_t M, int64_t ld,
                           const float* w, const pid_iso* iso, const pid_options* opt,
                           double* depth, double* in_in, double* in_out, int32_t* rank,
                           void* stream);

/*
 * pid_mean_weighted — PID-mean against a reliability-weighted mean contour (Sec. 4.1):
 * u_bar = sum_j c_j u_j with c_j = r_j / sum_k r_k, IN_in(i) = u_i subset_p u_bar and
 * IN_out(i) = u_bar subset_p u_i (the inclusions of Eq. 16), depth = min of the two.
 * data: soft masks [N][ld] (iso = NULL) or scalar fields mapped through `iso`.
 * member_weights: device float64 [N], r_j >= 0 and finite, not all zero; they are checked
 * on the device (a violation sets the domain bit reported by pid_sync, and the outputs are
 * zero). c_j is rounded to float32 once, and the mean contour's mass sum_j c_j m_j uses the
 * same rounded c_j, so the two inclusions refer to one mean contour. Equal weights give
 * pid_mean's results up to rounding. One streaming pass plus two small kernels; any
 * N <= 2^22.
 */
pid_status pid_mean_weighted(pid_handle h, const float* data, int64_t N, int64_t M, int64_t ld,
                             const float* w, const pid_iso* iso, const double* member_weights,
                             double* depth, double* in_in, double* in_out, int32_t* rank,
                             void* stream);

/*
 * pid_depth_from_matrix — PID (Eq. 10) from an inclusion matrix P[i][j] = u_i subset_p u_j
 * (Eq. 9; row-major FP64 [N][ldp] on the device, as pid_full's Gram modes return it),
 * optionally within groups of members. With labels (device int32 [N]; equal values = one
 * group), member i is compared only with the members of its own group C(i), which gives the
 * depth of i within its mode of a multimodal ensemble (Sec. 2.2):
 *   IN_in(i) = (1/|C(i)|) sum_{j in C(i)} P[i][j],  IN_out(i) = (1/|C(i)|) sum_{j in C(i)} P[j][i],
 *   depth = min, rank = position by depth within C(i) (0 = deepest; ties to the lower index).
 * labels = NULL: one group, i.e. the results pid_full computes from the same P. Outputs as
 * in pid_full (any may be NULL). 1 <= N <= 65536, ldp >= N. O(N^2) FP64 work, two kernels.
 */
pid_status pid_depth_from_matrix(pid_handle h, const double* P, int64_t N, int64_t ldp,
                                 const int32_t* labels, double* depth, double* in_in,
                                 double* in_out, int32_t* rank, void* stream);

/*
 * pid_spacetime — 4D (space-time) PID (Sec. 6.3): time is one more cell axis, so member i
 * is the function u_i(x, t) over the cells (x, t) of T time steps, and every sum over cells in
 * Eq. 6, 9, 14 and 15 runs over all T*M of them (the concatenation of the steps).
 * steps_host: HOST array of T device pointers, step t holding the members' values [N][ld]
 * at that time (soft masks, or fields mapped through `iso` when iso != NULL). w: cell measures [M],
 * the same at every step (a uniform time step cancels in every inclusion ratio), or NULL.
 * opt selects PID-mean, exact linear full PID or the tensor-core Gram as for pid_full
 * (NULL = PID-mean). The steps stay where they are (no copy into one array): they become
 * the descriptors of one persistent launch whose chunk partials are reduced by one
 * finalisation. N <= 512, 1 <= T <= 65536; all steps share
 * N, M and ld.
 */
pid_status pid_spacetime(pid_handle h, const float* const* steps_host, int32_t T, int64_t N,
                         int64_t M, int64_t ld, const float* w, const pid_iso* iso,
                         const pid_options* opt, double* depth, double* in_in, double* in_out,
                         int32_t* rank, double* P, double* err_est, void* stream);

/*
 * One ensemble of a batch. `data` are soft masks (is_field = 0) or scalar fields mapped
 * through `iso` (is_field = 1). Outputs as in pid_full; `mass` receives m_i and
 * `mean_depth` the PID-mean depth (both free by-products of every mode).
 */
typedef struct pid_ensemble {
  const float* data;
  int64_t N, M, ld;
  const float* w;           /* [M] or NULL */
  int32_t is_field;
  int32_t reserved;
  pid_iso iso;
  pid_options opt;
  double* depth;
  double* in_in;
  double* in_out;
  int32_t* rank;
  double* mass;
  double* mean_depth;
  double* P;                /* PID_MODE_FULL only */
  double* err_est;          /* PID_MODE_FULL only */
} pid_ensemble;

/*
 * pid_batch — many ensembles of uneven N and M in one persistent launch per kernel class,
 * the class launches recorded in order as one CUDA graph and replayed while the batch
 * layout is unchanged. Results are bitwise identical to the single-ensemble calls, with one
 * exception: a BF16 or split-BF16 Gram item (PID_MODE_FULL, up to 256 members) whose soft
 * masks are also those of a PID-mean or exact-full-PID item of the same batch (the same
 * data pointer, N, M, ld and cell measures) takes that item's exact PID-mean sums (m_i,
 * A_i of Eq. 16) instead of forming them in its own pass, so its IN_in is bitwise the
 * sibling's and its outputs differ from a single call only by the FP32 rounding of those
 * sums (below 1e-6). E4M3 items always take such sums from a streaming pass (their own
 * or an identical sibling's), which also yields their member scales. A PID-mean item over
 * the same data, cell measures and isovalue map as an exact-full-PID item of the batch
 * reads that item's first-pass partials instead of streaming the data again; those are
 * bitwise the partials its own pass would write, so this adds no exception.
 * Gram-mode ensembles of 257 to 512 members run the row-block-tiled Gram after their
 * class's streaming launch, one operand-staging and one tile launch each; they share one
 * operand buffer in the workspace, sized for the largest of them.
 */
pid_status pid_batch(pid_handle h, const pid_ensemble* ens, int32_t count, void* stream);

/*
 * Tile shapes. pid_autotune_shapes times, on the ensembles given (their data, shapes and
 * options, as for pid_batch), the tile choices that depend on the problem's shape, and keeps
 * the fastest per shape key (member count, cell-count octave, isovalue kind, cell measures;
 * for the Gram also the operand precision):
 *   - the streaming tile class: the default class (the first whose member rows hold N) and
 *     the next two larger ones (more member slots per warp, other cell widths);
 *   - the fused tensor-core Gram's cell chunk (one partial Gram per chunk): as planned,
 *     halved or doubled.
 * Each candidate runs once untimed and three times timed (CUDA events on `stream`; the call
 * synchronises it; not while the stream is being captured). Keys already tuned are kept.
 * Later single calls and batches on this handle plan with the chosen shapes, so a batch
 * stays bitwise equal to its single calls; a chosen shape changes the order of the FP32
 * sums (results move by FP32 rounding, within the stated bars). With PID_AUTOTUNE_CACHE set
 * the choices are appended to that file and loaded by later handles.
 */
pid_status pid_autotune_shapes(pid_handle h, const pid_ensemble* ens, int32_t count, void* stream);
/* Text of the handle's tuned entries (one per line) into buf (cap bytes, NUL-terminated);
 * returns the full length, or -1 for a NULL handle. */
int32_t pid_autotune_describe(pid_handle h, char* buf, int32_t cap);

/*
 * Serving. A server keeps ensembles resident on one GPU and answers depth requests that
 * arrive from any number of host threads. A scheduler thread forms batched steps from the
 * requests waiting at that moment and launches each step as one pid_batch on one of
 * `max_inflight` slots (each with its own stream and workspace) as soon as a slot is free,
 * so requests that arrive while others are on the GPU join the next step and steps overlap
 * on the device (continuous batching). A request's results do not depend on the requests
 * it is batched with: they are bitwise identical to a single call (the server's batches
 * never let a Gram request take a step-mate's sums).
 * Admission: ensembles are registered against an HBM budget; submissions beyond
 * max_queue are refused with PID_ERR_BUSY.
 */
typedef struct pid_serve_cfg {
  int32_t device;
  int32_t max_inflight;            /* concurrent steps (slots), >= 1 */
  int32_t max_batch;               /* requests per step, >= 1 */
  int32_t max_queue;               /* waiting requests before PID_ERR_BUSY, >= 1 */
  size_t hbm_budget_bytes;         /* resident ensembles + slot workspaces (0 = no cap) */
  size_t workspace_reserve_bytes;  /* per slot, counted against the budget */
  int64_t max_step_member_cells;   /* cap on sum N*M per step (0 = none) */
} pid_serve_cfg;

typedef struct pid_serve_stats {
  int64_t submitted, completed, failed, steps;
  double mean_batch;               /* requests per step */
  double p50_ms, p99_ms, max_ms;   /* submit -> results on the host */
  double requests_per_s;           /* completed / (last completion - first submit) */
  double member_cells_per_s;
  size_t resident_bytes;
} pid_serve_stats;

typedef struct pid_server_s* pid_server;

pid_status pid_serve_start(pid_server* out, const pid_serve_cfg* cfg);
/* Shut the server down in two steps.
 * pid_serve_cancel: the server takes no more requests (submit and register return
 *   PID_ERR_CANCELLED), queued requests complete with PID_ERR_CANCELLED, steps in flight
 *   finish, and every thread blocked in pid_serve_wait returns that request's status
 *   (PID_OK or PID_ERR_CANCELLED). Returns once the scheduler has exited. The handle stays
 *   valid: waits, stats and further cancels still work. Any thread may call it, any number
 *   of times.
 * pid_serve_stop: cancels (if not yet cancelled), waits until no thread is inside a
 *   pid_serve_* call on this server, then frees everything the server owns. The handle is
 *   invalid once it returns. Calls already inside the server when it is entered (a blocked
 *   wait, say) are safe; no new call may START once pid_serve_stop has been entered: join
 *   or quiesce other threads first (cancel, join, stop). */
pid_status pid_serve_cancel(pid_server s);
pid_status pid_serve_stop(pid_server s);
/* Register an ensemble [N][ld] float32 (soft masks, or fields with `iso`), cell measures w
 * [M] (or NULL). copy = 1: data (and w) are HOST pointers copied into device memory the
 * server owns; copy = 0: DEVICE pointers the caller keeps alive until pid_serve_unregister.
 * Either way its footprint counts against the budget (PID_ERR_OOM if it does not fit). */
pid_status pid_serve_register(pid_server s, const float* data, int64_t N, int64_t M, int64_t ld,
                              const float* w, int32_t is_field, const pid_iso* iso, int32_t copy,
                              int64_t* ensemble_id);
/* Replace the data of a server-owned ensemble (a new time step) from host memory; waits for
 * steps in flight that read it. */
pid_status pid_serve_update(pid_server s, int64_t ensemble_id, const float* data_host);
pid_status pid_serve_unregister(pid_server s, int64_t ensemble_id);
/* Queue a request; returns a ticket for pid_serve_wait. */
pid_status pid_serve_submit(pid_server s, int64_t ensemble_id, const pid_options* opt,
                            uint64_t* ticket);
/* Wait up to timeout_ms (< 0: forever) for a request; copies its results into the HOST
 * arrays given (any may be NULL; each N long) and retires the ticket. Returns the request's
 * status, or PID_ERR_TIMEOUT (ticket kept) if it is not done in time. */
pid_status pid_serve_wait(pid_server s, uint64_t ticket, int64_t timeout_ms, double* depth_host,
                          double* in_in_host, double* in_out_host, int32_t* rank_host,
                          double* mean_depth_host);
pid_status pid_serve_stats_get(pid_server s, pid_serve_stats* out);
pid_status pid_serve_stats_reset(pid_server s);

/*
 * pid_mean_noalloc — PID-mean (bitwise the result of pid_mean) for callers that cannot
 * allocate device memory: real-time loops in which a cudaMalloc would synchronise the
 * device, and host applications whose own allocator owns all device memory. The paper has
 * no counterpart; this is an interface convenience.
 *
 * No handle is needed and nothing is allocated: the scratch (per-chunk partial sums, FP64
 * totals, a finalisation ticket and an error word) lives in one fixed 4 MiB array inside
 * the library, which every GPU that loads the library holds until the process exits. The
 * caller still provides U (and w) and the outputs, all device pointers as for pid_mean.
 *
 * Limits: N <= 512 and 8 * (4 N + 2 N * n_chunks) + 256 bytes <= 4 MiB, where n_chunks is
 * the number of cell chunks the library splits M into (at most the device's SM count times
 * the members' group count, more only for very large M). Larger problems return
 * PID_ERR_UNSUPPORTED before anything is enqueued.
 *
 * The first call on a device (with that device current) performs a one-time set-up: it
 * looks up the device address of the scratch array and opts the kernels in to their shared
 * memory; make that first call before any stream capture. Later calls only enqueue work
 * on `stream`.
 *
 * The launch always takes the default column-sum exchange and ring depth of the streaming
 * kernel (no autotuning); every such choice sums in the same fixed order, so the outputs
 * equal pid_mean's bit for bit, tuned or not.
 *
 * There is no handle, so pid_last_error has no text for this call: the status alone says
 * what went wrong. PID_ERR_INVALID_ARG: N, M or ld out of range (N >= 1, M >= 1, ld >= M),
 * a null U, or no output. PID_ERR_UNSUPPORTED: N > 512, or the problem needs more scratch
 * than the fixed array holds (see Limits). PID_ERR_CUDA: the one-time set-up or a launch
 * failed.
 *
 * Every call on a device shares the one scratch array, which keeps the previous call's
 * contents; each call clears the parts that must start at zero. Calls whose work overlaps
 * on the GPU (different streams, or graphs replayed concurrently) race on the scratch and
 * produce wrong results: serialise them.
 *
 * device_status (device pointer to one uint32, may be NULL) receives the call's device
 * error word once the stream reaches it: 0 = success, bit 1 = a bounded device wait ran
 * out (the outputs are then not valid).
 */
pid_status pid_mean_noalloc(const float* U, int64_t N, int64_t M, int64_t ld, const float* w,
                            double* depth, double* in_in, double* in_out, int32_t* rank,
                            uint32_t* device_status, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PID_H_ */
