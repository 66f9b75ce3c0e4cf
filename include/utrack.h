/*
 * utrack.h — C ABI of the GB300 batched underwater-tracking environment.
 *
 * The library advances thousands of independent range-only tracking episodes
 * at once on one GPU: LRAUV heading kinematics, target motion, noisy
 * range-only pings, inter-agent communication, one particle filter per
 * (agent, target), observation tokens and reward, the transformer agent that
 * picks the next actions, and an optional learned range-only estimator.
 *
 * Paper: Gallici, Masmitja, Martin, "Scaling Multi-Agent Reinforcement
 * Learning for Underwater Acoustic Tracking via Autonomous Vehicles"
 * (arXiv 2505.08222).  Section references below are to that paper.
 *
 * Conventions for every entry point:
 *   - Return value: UT_OK or an error code; nothing throws across the ABI.
 *     env_last_error() describes the most recent error of a handle.
 *   - Asynchrony: every call is enqueued on the handle's CUDA stream and
 *     returns without waiting, except the ones documented as synchronising.
 *   - Pointers named *_dev are device pointers; *_host are host pointers.
 *     Device pointers returned by the library are borrowed: they stay valid
 *     until env_destroy() and their contents change with the next mutating
 *     call.  Caller-owned pointers are only read or written during the call
 *     (or, for device pointers, by the work the call enqueues).
 *   - Layouts: struct-of-arrays, float32 unless stated.  Agents, targets and
 *     filters of all environments are concatenated in environment order
 *     (CSR offsets from the per-environment counts).  Filter f of
 *     environment e, observer agent a, target k is
 *     f = filter_off[e] + a * T_e + k; particle i of filter f sits at
 *     f * n_particles + i (64-bit index).
 *   - A handle is not thread-safe.
 */
#ifndef UTRACK_H
#define UTRACK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define UT_ABI_VERSION 8u
#define UT_MAX_AGENTS 8      /* per environment */
#define UT_MAX_TARGETS 8     /* per environment */
#define UT_MAX_PARTICLES 4096
#define UT_TOKEN_FEATURES 8  /* observation token width */
#define UT_EST_RING 16       /* pings kept per filter for the learned estimator */
#define UT_EST_FEATURES 96   /* estimator input width (80 used, 16 zero) */

typedef enum {
  UT_OK = 0,
  UT_ERR_INVALID = 1,     /* bad argument or configuration */
  UT_ERR_NOMEM = 2,       /* allocation failed */
  UT_ERR_CUDA = 3,        /* CUDA runtime error (message in env_last_error) */
  UT_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
  UT_ERR_STATE = 5,       /* call not valid in the handle's current state */
  UT_ERR_UNSUPPORTED = 6  /* feature not available in this library or configuration */
} ut_status;

/* Caller-supplied device allocator.  alloc(bytes, stream, ctx) returns a
 * device pointer aligned to at least 256 bytes or NULL; free(ptr, stream,
 * ctx) releases it.  NULL allocator: the library uses cudaMallocAsync /
 * cudaFreeAsync on the handle's stream. */
typedef struct ut_allocator {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* ctx;
} ut_allocator;

/* Flags of ut_config.flags. */
#define UT_FLAG_DEBUG 1u       /* keep per-step intermediates (ut_debug_view) */
#define UT_FLAG_RING 2u        /* maintain the estimator ping ring every step */

/* Environment configuration (plain data, read at env_create only).
 * Constants of Sec. III-A.2 / III-A.3; the readings for what the paper leaves
 * open are the defaults documented per field. */
typedef struct ut_config {
  uint32_t abi_version;        /* must be UT_ABI_VERSION */
  uint32_t flags;              /* UT_FLAG_* */
  int32_t n_envs;              /* E >= 1 */
  int32_t max_agents;          /* 1..UT_MAX_AGENTS */
  int32_t max_targets;         /* 1..UT_MAX_TARGETS */
  int32_t n_particles;         /* P, 1..UT_MAX_PARTICLES, per filter */
  int32_t horizon;             /* episode length in steps (Termination paragraph) */
  const int32_t* agents_per_env_host;   /* [E] in 1..max_agents, or NULL: all max_agents */
  const int32_t* targets_per_env_host;  /* [E] in 1..max_targets, or NULL: all max_targets */
  float dt;                    /* step length, s (30 s, Sec. III-A.2) */
  float agent_speed;           /* m/s (1.0, Actions Space paragraph) */
  float heading_noise;         /* std of Gaussian heading noise, rad (0.02, Sec. III-A.3) */
  int32_t action_mode;         /* 0: {-turn, 0, +turn}; 1: equidistant rudder angles;
                                  2: rudder with adjacent moves (Sec. III-A.2 Actions Space):
                                  n_rudder equidistant angles, the agent's action moves its
                                  rudder one position down (0), keeps it (1) or moves it up (2),
                                  clamped at the ends; needs n_actions == 3 */
  int32_t n_rudder;            /* action_mode 2: rudder positions (5 in the paper), 2..8 */
  int32_t n_actions;           /* 3 for mode 0; 2..8 for mode 1 (7 default) */
  float turn_angle;            /* mode 0 heading change, rad */
  float rudder_max;            /* mode 1: rudder in [-rudder_max, rudder_max] (0.24 rad) */
  float rudder_gain;           /* mode 1: heading change = gain * rudder (1.45/0.24) */
  int32_t target_model;        /* 0: heading redrawn uniformly each step; 1: Gaussian drift */
  float target_speed_min, target_speed_max;  /* per-target speed drawn at reset, m/s */
  float target_drift_sigma;    /* model 1 heading increment std, rad */
  float target_depth_max;      /* target depth drawn in [0, max), m (0: surface) */
  float range_sigma;           /* range noise std, m */
  float det_radius;            /* pings heard iff 3-D distance <= det_radius, m */
  float comm_radius;           /* messages received iff distance <= comm_radius, m */
  float comm_drop;             /* probability that a message is dropped */
  float pf_accel_sigma;        /* particle velocity random-walk std per step, m/s */
  float pf_vcap;               /* particle speed cap, m/s */
  int32_t reward_type;         /* 0: tracking reward Eq. (1); 1: follow reward Eq. (2) */
  float eps_min, eps_max;      /* Eq. (1) errors, m (10, 50) */
  float follow_dmin;           /* Eq. (2) distance, m (50; 100 for fast targets) */
  float d_safe;                /* crash distance between agents, m */
  float spawn_min;             /* minimum spawn distance between entities, m (50) */
  float spawn_radius;          /* spawn disk radius, m (100 = half the 200 m maximum) */
  int32_t spawn_tries;         /* rejection-sampling tries per entity (64) */
  float feature_scale;         /* S: metres per unit in observation tokens */
  float est_scale;             /* L: metres per unit of the learned estimator's local frame (100) */
  /* Global index of this batch's first env / agent / target / filter when a
   * larger batch is split over several handles (one per GPU): random draws
   * are keyed by global ids, so the shards together reproduce the draws of
   * the whole batch.  0 for an unsplit batch. */
  uint32_t id_env0, id_agent0, id_target0, id_filter0;
  int32_t d_model;             /* transformer agent width; 0 = no policy */
  int32_t n_layers;            /* transformer blocks */
  int32_t n_heads;             /* attention heads (d_model % n_heads == 0) */
  /* 0: one filter per (env, agent, target) (Sec. III-A.2: every agent
   * tracks every target itself); 1: one filter per (env, target), fed every
   * ping of that target in the env (no communication limit), initialised
   * around the env's first agent, its estimate used by every agent. */
  int32_t shared_filter;
  /* Global index of this batch's first (agent, target) pair (pings are keyed
   * by pair); used with shared_filter = 1, where pairs and filters differ.
   * With per-agent filters a pair is its filter and id_filter0 applies. */
  uint32_t id_pair0;
  /* Resampling trigger: 0 resamples every step with a measurement (the
   * paper's filter); k in 1..16 carries the weights across steps as
   * per-particle log-weights and resamples only when the effective sample
   * size falls below k/16 of P.  The decision is exact integer arithmetic on
   * the max-normalised weights quantised to 15 bits, r = floor(w 2^15):
   * resample iff 16 (sum r)^2 < k P sum r^2. */
  int32_t pf_ess_num;
} ut_config;

typedef struct ut_env ut_env;

/* Borrowed device views of one step's outputs. */
typedef struct ut_step_out {
  const float* reward;       /* [E] shared reward (Eq. 1 or 2, normalised, -1 on crash) */
  const int32_t* done;       /* [E] 1 when the episode reached the horizon */
  const uint16_t* obs;       /* [NA][A_max+T_max][8] bf16 bit patterns */
  const float* estx;         /* [F] tracker estimate x */
  const float* esty;         /* [F] tracker estimate y */
  const float* err;          /* [F] 2-D tracking error of the estimate */
  const int32_t* actions;    /* [NA] actions applied this step */
  const float* logits;       /* [NA][n_actions] policy logits (NULL without policy) */
} ut_step_out;

/* Device views of the full environment state (struct of arrays). */
typedef struct ut_state_view {
  float *ax, *ay, *apsi;              /* agents [NA]; depth 0 */
  float *tx, *ty, *tz, *tpsi, *tspeed;/* targets [NT] */
  float *px, *py, *pvx, *pvy;         /* particles [F * P] */
  float *lpx, *lpy;                   /* last received pose of teammate b at agent a [NA * A_max] */
  int32_t* lpage;                     /* steps since that reception [NA * A_max] */
  float *estx, *esty;                 /* tracker estimates [F] */
  float *prev_estx, *prev_esty;       /* estimate before the last update [F] */
  float *prev2_estx, *prev2_esty;     /* estimate before that [F] */
  int32_t* rudder;                    /* rudder position per agent [NA] (action_mode 2) */
  float *velx, *vely;                 /* smoothed motion of the estimate per step [F]:
                                         v <- 0.85 v + 0.15 (e1 - e2) at every update */
  float* ring;                        /* estimator ring [F][16][4] (qx, qy, r, step) */
  int32_t *ring_head, *ring_count;    /* [F] */
  uint16_t* h;                        /* recurrent token bf16 [NA][d_model] (NULL without policy) */
  float* pw;                          /* particle log-weights [F * P], log w - max log w, 0 after a
                                         resample (NULL unless pf_ess_num > 0) */
  uint32_t step;                      /* global step counter g (random-stream position) */
  int32_t t_ep;                       /* steps since the last reset */
  int64_t n_agents, n_targets, n_filters; /* sizes, filled by env_get_state */
} ut_state_view;

/* Borrowed device views of per-step intermediates (UT_FLAG_DEBUG only). */
typedef struct ut_debug_view {
  /* (agent, target) pairs: sum over envs of A_e T_e, pair a T_e + k of env e
   * after the pairs of the earlier envs (the filter index with per-agent
   * filters) */
  float* range;        /* [pairs] noisy range heard by agent a of target k (0 if not heard) */
  int32_t* valid;      /* [pairs] detection bit */
  int32_t* recv;       /* [NA * A_max] agent a received agent b */
  float* meas;         /* [F][A_max][4] (qx, qy, qz, r) measurement list of each filter */
  int32_t* meas_n;     /* [F] */
  float *pred_px, *pred_py, *pred_pvx, *pred_pvy; /* [F * P] particles after predict */
  float* weight;       /* [F * P] normalised weights */
  float* wmax;         /* [F * P] exp(l_i - max l) */
  int32_t* idx;        /* [F * P] resample indices (identity without measurements) */
} ut_debug_view;

/* Statistics accumulated on the device since the last env_reset /
 * env_metrics_reset. */
typedef struct ut_rollout_stats {
  double sum_sq_err;       /* sum of squared 2-D tracking errors over filters and steps */
  int64_t n_err;           /* number of terms in sum_sq_err */
  double rmse;             /* sqrt(sum_sq_err / n_err) */
  double reward_sum;       /* sum over envs and steps */
  int64_t crash_count;     /* env-steps with a crash */
  int64_t agent_steps;     /* sum over steps of the number of agents */
  int64_t steps;           /* environment steps */
  int32_t device_status;   /* device error word (0 = none) */
  int64_t kernel_launches; /* kernels the library enqueued since the metrics were cleared */
} ut_rollout_stats;

/* Creates a handle and allocates every state buffer through `allocator`
 * (NULL: cudaMallocAsync).  `cuda_stream` (cudaStream_t, NULL = legacy
 * default stream) orders all later work of the handle.  Validates sizes:
 * counts within the maxima, 1 <= P <= UT_MAX_PARTICLES, d_model % n_heads.
 * Errors: UT_ERR_INVALID, UT_ERR_NOMEM, UT_ERR_CUDA.  On error *out is NULL. */
ut_status env_create(const ut_config* cfg, const ut_allocator* allocator, void* cuda_stream, ut_env** out);

/* Releases every buffer of the handle (after the stream's pending work). */
void env_destroy(ut_env* env);

/* Message of the most recent error of the handle ("" if none). */
const char* env_last_error(const ut_env* env);

/* Starts new episodes in every environment (Sec. III-A.2): agents on the
 * surface and targets spawned in a disk with pairwise separation >=
 * spawn_min (bounded rejection), first pings, each filter's particles
 * initialised around its agent at the heard range (uniform in the detection
 * disk if nothing was heard), recurrent tokens zeroed, observation tokens
 * of the reset state built, device metrics cleared.  The global step
 * counter becomes 0: every random draw is a function of (seed, step, ids). */
ut_status env_reset(ut_env* env, uint64_t seed);

/* One environment step, in order: actions -> agent kinematics
 * (Sec. III-A.3) -> target motion -> pings -> communication (Sec. III-A.2)
 * -> particle filter predict / weight / estimate / systematic resample
 * (Sec. II-A) -> observation tokens -> reward (Eq. 1 / Eq. 2).
 * actions_dev: [NA] int32 in [0, n_actions), or NULL: the transformer agent's
 * Gumbel-max sample when a policy is set, else uniform random actions.
 * out (optional): borrowed device views of this step's outputs. */
ut_status env_step(ut_env* env, const int32_t* actions_dev, ut_step_out* out);

/* T steps with policy (or random) actions, replayed from a captured CUDA
 * graph.  Clears the device metrics first; synchronises and fills `stats`
 * (host struct) with the metrics of these T steps.  T >= 1. */
ut_status rollout(ut_env* env, int32_t T, ut_rollout_stats* stats);

/* Captures and instantiates (and uploads) the T-step rollout graph without
 * running it, so that a later rollout(T) starts executing at once.  Not
 * synchronising. */
ut_status rollout_prepare(ut_env* env, int32_t T);

/* Stage timing.  When enabled, every eager env_step records a pair of CUDA
 * timing events on the launching stream around the tracker stage (the
 * particle filter, or the learned estimator in its place); graph rollouts
 * are not timed per stage (CUDA cannot time events recorded by graph nodes).
 * env_stage_time synchronises and returns the summed device time (ms) and the
 * number of timed stage launches since the previous read. */
ut_status env_profile(ut_env* env, int32_t enable);
ut_status env_stage_time(ut_env* env, double* total_ms, int64_t* launches);

/* Launch variants of the particle-filter step (threads per filter x
 * particles per thread).  Variant v is usable for P particles iff
 * pf_variant_usable(v, P); the handle starts with the default for its P and
 * the autotuner (bench / tests) may switch it.  Names are static strings. */
int32_t pf_variant_count(void);
int32_t pf_variant_usable(int32_t variant, int32_t P);
const char* pf_variant_label(int32_t variant);
ut_status env_set_pf_variant(ut_env* env, int32_t variant);
ut_status env_get_pf_variant(const ut_env* env, int32_t* variant);

/* Autotuner: times `reps` eager steps of every usable particle-filter variant
 * (CUDA events around the filter launches) and keeps the fastest; then, when
 * the handle qualifies for the persistent rollout (env_set_rollout_form),
 * times rollout(reps) in both forms with that variant and keeps the faster
 * form.  Both choices are recorded in a process-wide cache keyed by (n_envs,
 * max agents, max targets, P, filters); a later handle with the same key
 * takes the cached choices without timing.  The timed steps advance the
 * environment: call env_reset afterwards.  Synchronising.  *chosen
 * (optional) receives the variant. */
ut_status env_autotune(ut_env* env, int32_t reps, int32_t* chosen);

/* Rollout form used by rollout(T): 0 replays one captured CUDA graph of T
 * steps (every configuration); 1 runs one persistent kernel (Sec. III-A.3:
 * environments are independent, so one CTA advances one environment through
 * all T steps with block barriers only; an environment with one filter keeps
 * its particles in registers for the whole rollout).  Form 1 needs the
 * environment's uniform random actions (no policy set), the particle-filter
 * tracker (est_set_mode 0), every-step resampling (pf_ess_num 0) and a
 * filter variant that covers P, else UT_ERR_UNSUPPORTED; when the handle
 * stops qualifying (a policy or tracker mode set later), rollout() uses the
 * graph.  With the same filter variant both forms give the same state bit
 * for bit; the device metrics are the same sums in another order.
 * env_get_rollout_form reports the form rollout() would use now. */
ut_status env_set_rollout_form(ut_env* env, int32_t form);
ut_status env_get_rollout_form(const ut_env* env, int32_t* form);

/* Device views of the state buffers (borrowed).  Synchronises to read the
 * step counters. */
ut_status env_get_state(const ut_env* env, ut_state_view* out);

/* Copies state in from device pointers laid out as in ut_state_view; NULL
 * fields are left unchanged; step and t_ep are always taken. */
ut_status env_set_state(ut_env* env, const ut_state_view* in);

/* Device views of the last step's intermediates; UT_ERR_STATE unless the
 * handle was created with UT_FLAG_DEBUG. */
ut_status env_debug(const ut_env* env, ut_debug_view* out);

/* Synchronises and reads the device metrics (see ut_rollout_stats).
 * Returns UT_ERR_TIMEOUT when the device status word records a bounded wait
 * that gave up (status 2), UT_ERR_INVALID when it records a failed index
 * check of the checked build (status 3, library compiled with -DUT_CHECKED);
 * the stats are filled all the same.  env_metrics_reset clears the metrics
 * and the device status word. */
ut_status env_metrics(ut_env* env, ut_rollout_stats* out);
ut_status env_metrics_reset(ut_env* env);

/* Failure-detection test hook (no paper counterpart).  polls > 0: every
 * later launch of the handle's tensor-core kernels (transformer agent,
 * learned estimator) first waits on a barrier that nothing signals, gives up
 * after `polls` polls, and takes the same exit as a real timed-out wait:
 * device status word set, tensor memory freed, outputs of that launch not
 * written.  No copy or MMA is in flight when it gives up.  polls == 0
 * switches it off.  Captured rollout / collection graphs are re-captured.
 * Errors: UT_ERR_INVALID (null handle). */
ut_status env_test_wait_timeout(ut_env* env, uint32_t polls);

/* Transformer agent weights (Sec. III-B.1, Fig. 3; readings C16).  params_host
 * holds n_params floats in the canonical order: W_emb[d][8], b_emb[d]; per
 * block: ln1_g[d], ln1_b[d], Wqkv[3d][d], bqkv[3d], Wo[d][d], bo[d], ln2_g[d],
 * ln2_b[d], W1[4d][d], b1[4d], W2[d][4d], b2[d]; then lnf_g[d], lnf_b[d],
 * Wh[n_actions][d], bh[n_actions] (row-major, out x in).  Matrices are rounded
 * to BF16 (round to nearest even) and packed into tensor-core operand images;
 * vectors stay FP32.  Copied in (synchronising).  From then on env_step with
 * actions_dev == NULL and rollout() draw actions by the Gumbel-max rule from
 * the agent's logits on the previous observation.  Built for d_model 64 and
 * 128 with 16-wide heads (else UT_ERR_UNSUPPORTED); UT_ERR_STATE if the
 * handle was created with d_model == 0; UT_ERR_INVALID on a count mismatch. */
ut_status env_set_policy(ut_env* env, const float* params_host, int64_t n_params);

/* Transformer agent forward on caller buffers with the handle's weights:
 * tokens_dev [n_agents][n_slots][8] BF16 (16-byte aligned), n_slots in
 * 1 .. UT_MAX_AGENTS + UT_MAX_TARGETS, n_ent_dev [n_agents] entity tokens in
 * use (clamped to 0 .. n_slots), h_dev [n_agents][d_model] BF16 recurrent
 * embedding (16-byte aligned), read and replaced by the block output at the
 * recurrent token; logits_dev [n_agents][n_actions] FP32 written;
 * actions_dev [n_agents] (optional) receives Gumbel-max samples drawn at
 * global step `step`.  Errors: UT_ERR_STATE (no weights), UT_ERR_INVALID. */
ut_status policy_forward(ut_env* env, const uint16_t* tokens_dev, const int32_t* n_ent_dev, uint16_t* h_dev,
                         float* logits_dev, int32_t* actions_dev, int64_t n_agents, int32_t n_slots, uint32_t step,
                         void* cuda_stream);

/* ---------------------------------------------------------------------- */
/* Learned range-only estimator (no counterpart in the paper, whose tracker */
/* is the particle filter of Sec. II-A; readings C18).                     */
/* MLP 96 -> 256 -> 256 -> 256 -> 2, erf-GELU, a learned update of the      */
/* filter's estimate e1.  Features of a filter, in e1's local frame (units   */
/* of L = est_scale): its 16 most recent received pings, newest first, each */
/* [(q - e1)/L, (r - |q - e1|_3D)/L, (g - g_m)/16, 1], then the estimate's  */
/* last motion (e1 - e2)/L and smoothed motion v/L (v <- 0.85 v + 0.15      */
/* (e1 - e2) at each update), zero padded to 96 (FP32).  Output: the        */
/* correction (x - e1)/L; the new estimate is e1 + L * output, each output   */
/* clamped to +-3 in the step (the estimate is held when no ping arrived    */
/* this step).  Canonical                                                    */
/* order W1[256][96], b1, W2[256][256], b2, W3[256][256], b3, W4[2][256], b4 */
/* parameter order (156,930 floats).  Hidden layers on the tensor cores (BF16 */
/* FP32 accumulation; the first layer multiplies the features' BF16 high and */
/* low parts), FP32 master weights.                                          */
/* ---------------------------------------------------------------------- */
#define UT_EST_PARAMS 156930

typedef struct ut_est_train_config {
  int32_t steps;      /* Adam steps */
  int32_t batch;      /* rows per step, drawn uniformly with replacement
                         (batch == n_rows: the whole dataset in order) */
  float lr;           /* peak learning rate */
  int32_t cosine;     /* 1: cosine decay of lr to 0 over the steps */
  float beta1, beta2, eps;
  uint64_t seed;      /* batch sampling stream */
  float huber_delta;  /* 0: squared-error loss; > 0: Huber loss with this threshold (label units) */
} ut_est_train_config;

typedef struct ut_est_train_stats {
  double loss_first;  /* loss L of the first batch (definition at est_loss_grad) */
  double loss_last;   /* loss L of the last batch */
  double ms;          /* device time of the run */
  int64_t rows_seen;
} ut_est_train_stats;

/* Sets the FP32 weights (host, canonical order) and clears Adam's moments.
 * Synchronising.  Errors: UT_ERR_INVALID (count), UT_ERR_NOMEM, UT_ERR_CUDA. */
ut_status est_set_weights(ut_env* env, const float* params_host, int64_t n_params);
/* Copies the FP32 master weights out (synchronising). */
ut_status est_get_weights(ut_env* env, float* params_host, int64_t n_params);
/* 0: particle filter (default); 1-3: the learned estimator replaces the
 * filter stage of every step (needs weights and a handle created with
 * UT_FLAG_RING).  On a step without a fresh ping the estimate is held (1),
 * moved by the network all the same (2), or coasts by its smoothed motion v
 * (3, constant velocity; see ut_state_view.velx); with a fresh ping the
 * network's correction applies.  4: least-squares trilateration tracker
 * (Sec. II-A; Sec. III-A.2 names LS next to the PF) over the pings in each
 * filter's ring, the target taken as static over the window, depth known
 * (needs UT_FLAG_RING, no weights); the estimate is held with fewer than 3
 * pings or collinear senders (det A <= 1e-3 (tr A)^2 for the 2 x 2 normal
 * matrix A).  Errors: UT_ERR_INVALID (mode outside 0..4), UT_ERR_STATE. */
ut_status est_set_mode(ut_env* env, int32_t mode);
/* Raw network outputs out_dev [n_rows][2] of features X_dev [n_rows][96]. */
ut_status est_forward(ut_env* env, const float* X_dev, float* out_dev, int64_t n_rows);
/* Features [F][96] and labels [F][2] = (target - e1)/L of every filter's
 * last update (call after a step; e1, e2 = the estimates before it); needs
 * UT_FLAG_RING. */
ut_status est_record(ut_env* env, float* feat_dev, float* label_dev);
/* Loss of one batch of B rows of X_dev [n_rows][96], Y_dev [n_rows][2]
 * (device) and its gradient grad_dev [156930] (device, canonical order).
 * B == n_rows: the rows in order; otherwise B rows drawn uniformly with
 * replacement by the same counter-based stream as est_train's step `step`
 * under `seed` (so a loop of est_loss_grad + est_adam_step with est_train's
 * learning-rate schedule repeats est_train).  huber_delta == 0:
 * L = (1/(2B)) sum over rows and both outputs of (out - y)^2; > 0: the Huber
 * loss with that threshold (label units), (1/B) sum of the per-output loss.
 * Synchronising; *loss_host (optional) receives L.
 * Errors: UT_ERR_INVALID (sizes, B > 2^22, negative threshold),
 * UT_ERR_STATE (no weights), UT_ERR_NOMEM, UT_ERR_CUDA. */
ut_status est_loss_grad(ut_env* env, const float* X_dev, const float* Y_dev, int64_t n_rows, int32_t B,
                        uint64_t seed, uint32_t step, float huber_delta, float* grad_dev, double* loss_host);
/* One bias-corrected Adam update of the FP32 master weights with the given
 * gradient grad_dev [156930] (device; e.g. the average of the ranks'
 * est_loss_grad results in data-parallel training); the handle counts the
 * steps for the bias correction (reset by est_set_weights / est_load).
 * lr >= 0 (a cosine schedule ends at 0: the moments still advance), beta1
 * and beta2 in [0, 1), eps > 0.  Asynchronous on the handle's stream.
 * Errors: UT_ERR_INVALID, UT_ERR_STATE. */
ut_status est_adam_step(ut_env* env, const float* grad_dev, float lr, float beta1, float beta2, float eps);
/* Adam (bias-corrected) over cfg->steps batches of X_dev / Y_dev
 * ([n_rows][96], [n_rows][2], device).  Synchronising; stats optional. */
ut_status est_train(ut_env* env, const float* X_dev, const float* Y_dev, int64_t n_rows,
                    const ut_est_train_config* cfg, ut_est_train_stats* stats);
/* Raw little-endian file: 4 uint32 header (magic, version, count, Adam step),
 * then FP32 master weights, first and second moments. */
ut_status est_save(ut_env* env, const char* path);
ut_status est_load(ut_env* env, const char* path);

/* ---------------------------------------------------------------------- */
/* Stand-alone operations (the same device code the step uses).            */
/* ---------------------------------------------------------------------- */

/* Philox4x32-10 of n counters: ctr_dev [n][4] uint32, key = seed (low word
 * first), out_dev [n][4].  Errors: UT_ERR_INVALID (n < 0), UT_ERR_CUDA. */
ut_status ut_philox(const uint32_t* ctr_dev, uint64_t seed, uint32_t* out_dev, int64_t n, void* cuda_stream);

/* Systematic resampling (Sec. II-A; readings C4, C5) of n_filters filters of
 * P particles: wmax_dev [n_filters][P] holds exp(l_i - max l) in [0, 1] with
 * at least one entry equal to 1; u64_dev [n_filters] the random offset bits.
 * With q_i = floor(w_i 2^38), Q the inclusive sum, W = Q[P-1] and
 * U0 = floor(u64 W / 2^64): idx[j] = min{ i : P Q_i > j W + U0 }.
 * Writes idx_dev [n_filters][P] int32.  Errors: UT_ERR_INVALID, UT_ERR_CUDA. */
ut_status pf_resample(const float* wmax_dev, const uint64_t* u64_dev, int64_t n_filters, int32_t P,
                      int32_t* idx_dev, void* cuda_stream);

/* BF16 GEMM on the tensor cores (tcgen05.mma, FP32 accumulation in tensor
 * memory): C[M][N] = A[M][K] * B[N][K]^T, row-major, A and B BF16 bit
 * patterns (16-byte aligned), C FP32.  16 <= N <= 256 and 16 <= K <= 256, both
 * multiples of 16; any M >= 1.  The primitive the transformer agent (Sec.
 * III-B.1, Fig. 3) and the estimator are built from, exposed on its own.
 * status_dev (optional, device int32) receives 4 if a bounded wait for the
 * tensor core gave up.  Errors: UT_ERR_INVALID, UT_ERR_CUDA. */
ut_status tc_gemm_bf16(const uint16_t* A_dev, const uint16_t* B_dev, float* C_dev, int32_t M, int32_t N, int32_t K,
                       int32_t* status_dev, void* cuda_stream);

/* ---------------------------------------------------------------------- */
/* Allocation-free tracker update (the paper has no counterpart).          */
/* ---------------------------------------------------------------------- */

/* For callers that must not allocate device memory: real-time host threads
 * that forbid allocator calls (an allocation may synchronise the device and
 * take unbounded time), a vehicle simulator that owns every buffer and the
 * GPU's memory budget, or a plug-in whose host process has handed all device
 * memory to another framework's pool.  It runs the tracking part of one step
 * on caller buffers: pings and communication at the given (already moved)
 * agent and target positions, then the particle-filter step (predict,
 * weight, estimate, systematic resample) of every (env, agent, target)
 * filter — the same rules and random draws as env_step at global step
 * `step` (>= 1) with `seed`, including the global id offsets cfg->id_env0,
 * id_agent0, id_target0 and id_filter0 of a sharded batch.  Uniform fleets
 * only: cfg->n_envs environments of cfg->max_agents agents and
 * cfg->max_targets targets (the per-env count pointers must be NULL),
 * per-agent filters resampled every step (shared_filter and pf_ess_num 0);
 * cfg supplies the constants.
 *   ax/ay_dev [E*A], tx/ty/tz_dev [E*T]: positions (read);
 *   px/py/pvx/pvy_dev [E*A*T*P]: particles, updated in place; 16-byte
 *     aligned when P % 4 == 0 (read and written as float4), else
 *     UT_ERR_INVALID;
 *   estx/esty/err_dev [E*A*T]: estimate and its 2-D error (written).
 * Intermediates (layout tables, per-filter measurement lists) live in a
 * static device array of about 5.1 MB that every GPU loading the library
 * holds until exit; the call itself allocates nothing (no cudaMalloc, no
 * allocator callback).  Limit: at most 8192 environments and 32768 filters
 * (E*A*T) per call; larger sizes return UT_ERR_INVALID with a message on
 * stderr.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array: calls that overlap on the GPU race.  Enqueued on
 * cuda_stream, not synchronising.  Errors: UT_ERR_INVALID, UT_ERR_CUDA. */
ut_status tracker_update_noalloc(const ut_config* cfg, uint64_t seed, uint32_t step, const float* ax_dev,
                                 const float* ay_dev, const float* tx_dev, const float* ty_dev, const float* tz_dev,
                                 float* px_dev, float* py_dev, float* pvx_dev, float* pvy_dev, float* estx_dev,
                                 float* esty_dev, float* err_dev, void* cuda_stream);

/* ---------------------------------------------------------------------- */
/* TransfMAPPO training (Sec. II-B: MAPPO, PPO's clipped surrogate for the  */
/* actors and one centralized critic V(S) on the global state; Sec. III-B.1 */
/* and Fig. 3: TransformerAgent and TransformerCritic, one architecture,    */
/* the critic fed the true position, velocity and heading of every entity   */
/* and keeping its own recurrent embedding).                               */
/*                                                                          */
/* A ut_tfm handle holds one transformer in FP32 for training — the actor  */
/* (n_out = n_actions, same parameter layout as env_set_policy) or the      */
/* critic (n_out = 1) — with its Adam moments and the activation buffers of */
/* up to max_batch samples.  A sample is n_slots entity tokens of 8 values  */
/* (the first n_ent of them in use) plus a recurrent embedding h of d_model */
/* floats at token 0; the network is the agent's (pre-LN blocks, FFN 4d     */
/* with erf-GELU, LayerNorm epsilon 1e-5, final LayerNorm and a linear head */
/* on token 0).  Readings: the recurrent input is data (no backpropagation  */
/* through time); PPO per sample L = -min(r A, clip(r, 1-eps, 1+eps) A)     */
/* - ent_coef H(pi) with r = exp(log pi(a) - log pi_old(a)) (Schulman et    */
/* al. 2017, Eq. 7 and 9); value loss (V - R)^2; batch losses are means.    */
/* Calls are enqueued on the handle's stream; those that return statistics */
/* to a host pointer synchronise.  Not thread-safe.                         */
/* ---------------------------------------------------------------------- */
typedef struct ut_tfm ut_tfm;

typedef struct ut_tfm_config {
  uint32_t abi_version;  /* must be UT_ABI_VERSION */
  int32_t d_model;       /* 32, 64, 96 or 128 */
  int32_t n_layers;      /* 1 .. 8 */
  int32_t n_heads;       /* head width d_model / n_heads in {8, 16, 32} */
  int32_t n_out;         /* 1 .. 16 head outputs */
  int32_t n_slots;       /* entity token slots per sample, 1 .. UT_MAX_AGENTS + UT_MAX_TARGETS */
  int32_t tokens_bf16;   /* 1: tokens are BF16 (the observation tokens), 0: FP32 */
  int32_t reserved;
  int64_t max_batch;     /* samples per call, 1 .. 2^22 */
} ut_tfm_config;

/* Number of parameters of the configuration (canonical order of
 * env_set_policy with n_actions = n_out), or -1 if it is invalid. */
int64_t tfm_param_count(const ut_tfm_config* cfg);

/* Creates the handle on cuda_stream with a copy of params_host (n_params
 * floats, canonical order) as the FP32 master weights and zero Adam moments.
 * Device memory: about (16 d + 8) x 4 bytes per token row per block plus
 * the backward buffers, for max_batch x (1 + n_slots) rows.
 * Errors: UT_ERR_INVALID (configuration or count), UT_ERR_NOMEM, UT_ERR_CUDA. */
ut_status tfm_create(const ut_tfm_config* cfg, const float* params_host, int64_t n_params, void* cuda_stream,
                     ut_tfm** out);
void tfm_destroy(ut_tfm* t);
const char* tfm_last_error(const ut_tfm* t);

/* Borrowed device pointer to the FP32 master weights (n_params floats),
 * valid until tfm_destroy; writes through it change the network. */
ut_status tfm_params(ut_tfm* t, float** params_dev);

/* GEMM path of the handle's forward and backward (the dense contractions of
 * the linear layers): 1 (default) BF16 operands on the tensor cores
 * (tcgen05.mma, FP32 accumulation in tensor memory; activations stay FP32 in
 * memory and are rounded to BF16 as they are staged); 0 FP32 on the CUDA
 * cores.  Attention, LayerNorm, losses and reductions are FP32 either way.
 * A bounded tensor-core wait that gave up is reported as UT_ERR_TIMEOUT by
 * the next call that returns statistics.  Errors: UT_ERR_INVALID. */
ut_status tfm_set_gemm_path(ut_tfm* t, int32_t tensor_cores);

/* Forward of n samples (1 .. max_batch).  Sample s reads batch row
 * b = sel_dev ? sel_dev[s] : s of: tokens_dev [.][n_slots][8] (FP32, or BF16
 * when tokens_bf16), n_ent_dev [.] (clamped to 0 .. n_slots) and h_dev
 * [.][d_model] FP32.  Writes out_dev [n][n_out] and, if h_out_dev is not
 * NULL, h_out_dev [n][d_model] = the residual stream at token 0 after the
 * last block (the next recurrent embedding).  h_out_dev may equal h_dev
 * when sel_dev is NULL.  Errors: UT_ERR_INVALID, UT_ERR_CUDA. */
ut_status tfm_forward(ut_tfm* t, const void* tokens_dev, const int32_t* n_ent_dev, const float* h_dev,
                      const int32_t* sel_dev, int64_t n, float* out_dev, float* h_out_dev);

/* PPO actor loss over n samples (rows selected as in tfm_forward) and its
 * gradient: actions_dev [.] in 0 .. n_out-1, logp_old_dev [.] the behaviour
 * policy's log-probability of the action, adv_dev [.] advantages;
 * clip_eps > 0, ent_coef >= 0.  grad_dev [n_params] is overwritten with the
 * gradient of the mean loss.  stats_host (optional; NULL keeps the call
 * asynchronous) receives the means of [loss, entropy, clipped fraction
 * (|r - 1| > eps), log pi_old - log pi].  Errors: UT_ERR_INVALID (also for
 * a handle with n_out < 2), UT_ERR_CUDA. */
ut_status tfm_ppo_actor_grad(ut_tfm* t, const void* tokens_dev, const int32_t* n_ent_dev, const float* h_dev,
                             const int32_t* sel_dev, int64_t n, const int32_t* actions_dev,
                             const float* logp_old_dev, const float* adv_dev, float clip_eps, float ent_coef,
                             float* grad_dev, double* stats_host);

/* Critic loss mean (V - R)^2 over n samples against returns_dev [.] and its
 * gradient (grad_dev [n_params], overwritten).  stats_host (optional)
 * receives the means of [loss, V, 0, 0].  Errors: UT_ERR_INVALID (also for a
 * handle with n_out != 1), UT_ERR_CUDA. */
ut_status tfm_value_grad(ut_tfm* t, const void* tokens_dev, const int32_t* n_ent_dev, const float* h_dev,
                         const int32_t* sel_dev, int64_t n, const float* returns_dev, float* grad_dev,
                         double* stats_host);

/* One Adam step (Kingma & Ba 2015, Algorithm 1, with bias correction) on the
 * master weights from grad_dev [n_params]: lr >= 0, beta1 and beta2 in
 * [0, 1), eps > 0.  Errors: UT_ERR_INVALID, UT_ERR_CUDA. */
ut_status tfm_adam_step(ut_tfm* t, const float* grad_dev, float lr, float beta1, float beta2, float eps);

/* Copies the actor's master weights into env's transformer agent (as
 * env_set_policy: matrices rounded to BF16 and packed); the configuration
 * must match the env's (d_model, n_layers, n_heads, n_out = n_actions).
 * Synchronises both streams.  Errors: UT_ERR_INVALID, UT_ERR_STATE,
 * UT_ERR_UNSUPPORTED (as env_set_policy), UT_ERR_CUDA. */
ut_status tfm_sync_policy(ut_tfm* t, ut_env* env);

/* Generalized advantage estimation (Schulman et al. 2016, Eq. 16) by the
 * backward recursion A_t = delta_t + gamma lambda (1 - done_t) A_{t+1},
 * delta_t = r_t + gamma (1 - done_t) V_{t+1} - V_t, and R_t = A_t + V_t:
 * reward_dev, done_dev [T][E] (done_t = 1 when step t ended an episode),
 * value_dev [T+1][E] (the last row bootstraps); adv_dev, ret_dev [T][E].
 * If agent_env_dev [NA] (the env of each agent) and adv_agent_dev [T][NA]
 * are given, the env's advantage is also written for each of its agents.
 * FP32 arithmetic, one thread per env.  Enqueued on cuda_stream.
 * Errors: UT_ERR_INVALID, UT_ERR_CUDA. */
ut_status ppo_gae(const float* reward_dev, const float* value_dev, const int32_t* done_dev, int32_t T, int64_t E,
                  float gamma, float lam, float* adv_dev, float* ret_dev, const int32_t* agent_env_dev, int64_t NA,
                  float* adv_agent_dev, void* cuda_stream);

/* Critic tokens of every env from the true state (Sec. III-A: the global
 * state holds the true 3-D position, velocity and direction of each
 * entity): tokens_dev [E][A_max + T_max][8] FP32, agents then targets packed
 * from slot 0, each [x/S, y/S, z/S, vx, vy, cos psi, sin psi, kind] with S =
 * feature_scale, velocity in m/s (agents at depth 0 moving at agent_speed)
 * and kind 1 for an agent, 0 for a target; zero padding; n_ent_dev [E] =
 * A_e + T_e.  Enqueued on the env's stream.  Errors: UT_ERR_INVALID. */
ut_status env_state_tokens(ut_env* env, float* tokens_dev, int32_t* n_ent_dev);

/* Rollout recording for the PPO batch, on the env's stream.
 * env_ppo_snapshot, before env_step: the agents' current observation
 * tokens (the policy's input) to tokens_dev [NA][A_max + T_max][8] BF16,
 * their entity counts to n_ent_dev [NA] and the recurrent embedding (BF16)
 * to h_dev [NA][d_model] FP32.  env_ppo_record, after an env_step whose
 * actions the transformer agent drew: actions_dev [NA], logp_dev [NA] =
 * log-softmax of the agent's logits at its action, reward_dev [E],
 * done_dev [E].  Each pointer may be NULL (not recorded).
 * Errors: UT_ERR_STATE (no transformer agent), UT_ERR_INVALID, UT_ERR_CUDA. */
ut_status env_ppo_snapshot(ut_env* env, uint16_t* tokens_dev, int32_t* n_ent_dev, float* h_dev);
ut_status env_ppo_record(ut_env* env, int32_t* actions_dev, float* logp_dev, float* reward_dev, int32_t* done_dev);

/* Device buffers of one PPO collection of T steps (all on the env's GPU;
 * NA agents, E envs, NS = A_max + T_max slots, d the agent's d_model, dc the
 * critic's): tokens [T][NA][NS][8] BF16, n_ent [T][NA], h [T][NA][d],
 * actions [T][NA], logp [T][NA], reward [T][E], done [T][E] (as
 * env_ppo_snapshot / env_ppo_record), ctokens [T+1][E][NS][8] FP32 and
 * cn_ent [T+1][E] (as env_state_tokens), ch [T+2][E][dc] the critic's
 * recurrent embedding (ch[0] read: the caller sets it, zero at an episode
 * start; ch[t+1] written from the forward at t), value [T+1][E]. */
typedef struct ut_ppo_buffers {
  uint16_t* tokens;
  int32_t* n_ent;
  float* h;
  int32_t* actions;
  float* logp;
  float* reward;
  int32_t* done;
  float* ctokens;
  int32_t* cn_ent;
  float* ch;
  float* value;
} ut_ppo_buffers;

/* T collection steps as one CUDA graph (captured on first use, reused while
 * the arguments and the env's step configuration stay the same): for t = 0 ..
 * T-1 the critic tokens and forward at t, the snapshot, one env_step with the
 * transformer agent acting and the record; then the critic at T (the
 * bootstrap value).  The same kernels and results as the sequence of the
 * separate calls.  critic: a ut_tfm with n_out 1, FP32 tokens, n_slots = NS
 * and max_batch >= E; its activation buffers are used by the graph, which
 * starts after the work already enqueued on the env's stream, so work on the
 * critic handle must be ordered with that stream (create it on the env's
 * stream).  The graph reads the weights at run time: later weight updates
 * (tfm_adam_step, env_set_policy) are seen without a new capture.  Enqueued
 * on the env's stream.  Errors: UT_ERR_INVALID, UT_ERR_STATE (no env_reset or
 * no agent weights), UT_ERR_CUDA. */
ut_status env_ppo_collect(ut_env* env, ut_tfm* critic, int32_t T, const ut_ppo_buffers* buffers);

#ifdef __cplusplus
}
#endif

#endif /* UTRACK_H */
