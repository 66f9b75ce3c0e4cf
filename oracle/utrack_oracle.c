/*
 * FP64 CPU oracle for the batched underwater-tracking environment step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * restatement of the method that the CUDA path is checked against.  It shares
 * no code, header, table or constant generator with the CUDA library.  Only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg load it.
 *
 * Method (Gallici, Masmitja, Martin, "Scaling Multi-Agent Reinforcement
 * Learning for Underwater Acoustic Tracking via Autonomous Vehicles"):
 *   - spawn / step timing / per-agent per-target trackers: Sec. III-A.2
 *     ("PyLrauv UTracking Environment");
 *   - observation space, reward (Eq. 1 tracking, Eq. 2 follow, target
 *     normalisation, crash penalty), action space, termination: the
 *     paragraphs of Sec. III-A.2;
 *   - heading kinematics p' = p + v dt [cos(psi+dpsi), sin(psi+dpsi)], the
 *     linear rudder-to-heading map and 0.02 rad heading noise: Sec. III-A.3
 *     ("JaxLrauv UTracking");
 *   - particle filter (weighted particles moved by a motion model, weighted
 *     by measurement likelihoods, resampled): Sec. II-A;
 *   - transformer agent (entity tokens + recurrent token, self-attention,
 *     LayerNorm, MLP head on the recurrent token): Sec. III-B.1, Fig. 3.
 * Where the paper is silent a reading is taken (numbered C1-C23 where it is
 * used below); every such constant is a field of oc_config.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), keyed by the seed, counter =
 * (id0, id1, global step, stream tag).  The CUDA side implements the same
 * published generator separately.
 *
 * Parity pins (tests/test_oracle_*.py): Philox bijectivity and statistics,
 * straight-line and circular kinematics closed forms, noise-free ranges equal
 * Euclidean distance, weights sum to one and are shift invariant, brute-force
 * Bayes and brute-force systematic resampling on tiny particle sets,
 * trilateration convergence of the whole filter, Eq. 1 / Eq. 2 printed values,
 * transformer permutation invariance and a hand-derived one-token case, MLP
 * gradients against central finite differences, Adam against its closed form
 * on a constant gradient.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OC_MAX_AGENTS 8
#define OC_MAX_TARGETS 8
#define OC_MAX_MEAS OC_MAX_AGENTS
#define OC_RING 16
#define OC_FEAT 96
#define OC_VEL_KEEP 0.85 /* smoothing of the estimate motion (reading C18) */
#define OC_TOKEN 8

/* Philox stream tags (counter word 3). */
enum {
  OC_TAG_SPAWN = 1,
  OC_TAG_AGENT_INIT = 2,
  OC_TAG_TARGET_INIT = 3,
  OC_TAG_PF_INIT = 4,
  OC_TAG_PF_INIT2 = 5,
  OC_TAG_ACTION = 6,
  OC_TAG_AGENT_NOISE = 7,
  OC_TAG_TARGET_MOVE = 8,
  OC_TAG_PING = 9,
  OC_TAG_COMM = 10,
  OC_TAG_PF_PREDICT = 11,
  OC_TAG_RESAMPLE = 12,
  OC_TAG_GUMBEL = 13,
  OC_TAG_RESET_PING = 15
};

typedef struct {
  int32_t n_envs, max_agents, max_targets, n_particles;
  const int32_t *agent_off, *target_off, *filter_off; /* [n_envs+1] */
  double dt, agent_speed, heading_noise;
  int32_t action_mode; /* 0: {-turn,0,+turn}; 1: rudder angles; 2: rudder, adjacent moves */
  int32_t n_rudder;    /* action_mode 2: rudder positions */
  int32_t n_actions;
  double turn_angle, rudder_max, rudder_gain;
  int32_t target_model; /* 0: heading redrawn each step; 1: heading drift */
  double target_speed_min, target_speed_max, target_drift_sigma, target_depth_max;
  double range_sigma, det_radius, comm_radius, comm_drop;
  double pf_accel_sigma, pf_vcap;
  int32_t reward_type; /* 0: tracking Eq. 1; 1: follow Eq. 2 */
  double eps_min, eps_max, follow_dmin, d_safe;
  double spawn_min, spawn_radius;
  int32_t spawn_tries;
  double feature_scale;
  uint64_t seed;
  /* Global index of this batch's first env / agent / target / filter in a
   * larger batch: random draws are keyed by global ids, so a sub-batch of
   * independent environments replays exactly the draws of the full batch. */
  int32_t env0, agent0, target0, filter0;
  double est_scale; /* L: local frame of the learned estimator's features */
  /* 0: one filter per (env, agent, target), filter a T + k of the env;
   * 1: one filter per (env, target), filter k, fed every ping of the target
   * and anchored at the env's first agent (reading C22). */
  int32_t shared_filter;
  /* Global index of the first (agent, target) pair: pings are keyed by pair
   * (pair a T + k of env e after pair_off[e]); with per-agent filters the
   * pairs are the filters and filter0 applies. */
  int32_t pair0;
  const int32_t* pair_off; /* [n_envs+1] */
  /* Resampling trigger (reading C23): 0 resamples every step with a
   * measurement; k in 1..16 carries log-weights across steps and resamples
   * iff 16 (sum r)^2 < k P sum r^2, r = floor(w 2^38) >> 23. */
  int32_t pf_ess_num;
} oc_config;

typedef struct {
  double *ax, *ay, *apsi;                   /* agents  [NA] (z = 0, surface) */
  double *tx, *ty, *tz, *tpsi, *tspeed;     /* targets [NT] */
  double *px, *py, *pvx, *pvy;              /* particles [F*P] */
  double *lpx, *lpy;                        /* last received teammate pose [NA*A_max] */
  int32_t *lpage;                           /* steps since last reception [NA*A_max] */
  double *estx, *esty;                      /* tracker estimate [F] */
  double *prev_estx, *prev_esty;            /* estimate before the last update [F] */
  double *prev2_estx, *prev2_esty;          /* estimate before that [F] */
  double *velx, *vely;                      /* smoothed motion of the estimate [F] */
  int32_t *rudder;                          /* rudder position per agent [NA] (action_mode 2) */
  double *ring;                             /* [F*16*4]: qx, qy, r, step */
  int32_t *ring_head, *ring_count;          /* [F] */
  uint32_t step;                            /* global step counter g */
  int32_t t_ep;                             /* steps since reset */
  double *pw;                               /* particle log-weights [F*P] (pf_ess_num > 0) */
} oc_state;

/* Per-step outputs and intermediates, all optional (NULL = not wanted). */
typedef struct {
  double *range;          /* [pairs] noisy range of target k at agent a */
  int32_t *valid;         /* [pairs] detection bit */
  int32_t *recv;          /* [NA*A_max] a received b this step */
  double *meas;           /* [F*A_max*4] qx, qy, qz, r */
  int32_t *meas_n;        /* [F] */
  double *pred_px, *pred_py, *pred_pvx, *pred_pvy; /* [F*P] after predict */
  double *weight;         /* [F*P] normalised weights */
  double *wmax;           /* [F*P] max-normalised weights exp(l - max l) */
  int32_t *idx;           /* [F*P] resample indices (identity when no update) */
  double *err;            /* [F] tracking error */
  double *tokens;         /* [NA*(A_max+T_max)*8] */
  double *reward;         /* [E] */
  int32_t *crash;         /* [E] */
} oc_step_out;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11).  Round: two 32x32->64 products of counter words 0  */
/* and 2 with the published multipliers; the high halves are xored with the */
/* other counter words and the round key; key bumped by the Weyl constants. */
/* ------------------------------------------------------------------------ */
void oc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint32_t id0, uint32_t id1, uint32_t step, uint32_t tag, uint32_t out[4]) {
  uint32_t ctr[4] = {id0, id1, step, tag};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  oc_philox4x32_10(ctr, key, out);
}

/* Uniform on [0,1) with 24 random bits (exact in float and double). */
static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }
/* Uniform on (0,1]. */
static double u01_open_low(uint32_t x) { return (double)((x >> 8) + 1u) * (1.0 / 16777216.0); }
/* Uniform on (0,1), cell midpoints. */
static double u01_mid(uint32_t x) { return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0); }

/* Box-Muller: two independent standard normals from two uniforms. */
static void normal_pair(uint32_t xa, uint32_t xb, double* n0, double* n1) {
  double r = sqrt(-2.0 * log(u01_open_low(xa)));
  double th = 2.0 * M_PI * u01(xb);
  *n0 = r * cos(th);
  *n1 = r * sin(th);
}

void oc_uniform_normal(uint64_t seed, uint32_t id0, uint32_t id1, uint32_t step, uint32_t tag,
                       double out_u[4], double out_n[4]) {
  uint32_t x[4];
  draw(seed, id0, id1, step, tag, x);
  for (int i = 0; i < 4; ++i) out_u[i] = u01(x[i]);
  normal_pair(x[0], x[1], &out_n[0], &out_n[1]);
  normal_pair(x[2], x[3], &out_n[2], &out_n[3]);
}

/* Wrap an angle to [-pi, pi). */
static double wrap_angle(double a) { return a - 2.0 * M_PI * floor((a + M_PI) / (2.0 * M_PI)); }

/* Heading change of action j.  Mode 0: {-turn, 0, +turn}.  Mode 1: rudder
 * angle gamma_j equidistant in [-rudder_max, rudder_max] and the linear map
 * dpsi = theta(gamma) = rudder_gain * gamma (Sec. III-A.3; the Actions Space
 * paragraph fixes +-0.24 rad rudder <-> +-1.45 rad heading at 1 m/s, 30 s).
 * Mode 2 (the Actions Space paragraph's rudder that moves only to an
 * adjacent angle): j is the rudder position reached, out of n_rudder. */
static double action_dpsi(const oc_config* c, int32_t j) {
  if (c->action_mode == 0) return (double)(j - 1) * c->turn_angle;
  int n = c->action_mode == 2 ? c->n_rudder : c->n_actions;
  double gamma = -c->rudder_max + 2.0 * c->rudder_max * (double)j / (double)(n - 1);
  return c->rudder_gain * gamma;
}

static int32_t env_agents(const oc_config* c, int e) { return c->agent_off[e + 1] - c->agent_off[e]; }
static int32_t env_targets(const oc_config* c, int e) { return c->target_off[e + 1] - c->target_off[e]; }
/* The filter agent a of env e uses for target k. */
static int32_t filter_index(const oc_config* c, int e, int a, int k) {
  return c->filter_off[e] + (c->shared_filter ? k : a * env_targets(c, e) + k);
}
/* Filters of env e, and the anchor agent and target of its j-th filter. */
static int32_t env_filters(const oc_config* c, int e) { return c->filter_off[e + 1] - c->filter_off[e]; }
static int32_t filter_agent(const oc_config* c, int e, int j) { return c->shared_filter ? 0 : j / env_targets(c, e); }
static int32_t filter_target(const oc_config* c, int e, int j) { return c->shared_filter ? j : j % env_targets(c, e); }
/* (agent, target) pair of env e, and the global key of its pings. */
static int32_t pair_index(const oc_config* c, int e, int a, int k) {
  return c->pair_off[e] + a * env_targets(c, e) + k;
}
static uint32_t pair_key(const oc_config* c, int32_t p) {
  return (uint32_t)((c->shared_filter ? c->pair0 : c->filter0) + p);
}

/* ------------------------------------------------------------------------ */
/* Reset (Sec. III-A.2): agents on the surface, targets at a random depth,  */
/* every pair of entities at least spawn_min apart, all inside a disk of    */
/* radius spawn_radius = spawn_max / 2 (so no pair is farther than          */
/* spawn_max).  Bounded rejection on a 2^-16 m integer lattice so that the  */
/* accept/reject decision is exact integer arithmetic; after spawn_tries    */
/* failures the last candidate inside the disk is kept (reading C13).       */
/* ------------------------------------------------------------------------ */
static void spawn_env(const oc_config* c, int e, uint32_t g, double* ex, double* ey) {
  int n_ent = env_agents(c, e) + env_targets(c, e);
  int64_t X[OC_MAX_AGENTS + OC_MAX_TARGETS], Y[OC_MAX_AGENTS + OC_MAX_TARGETS];
  const double q = 65536.0;
  int64_t r_int = (int64_t)floor(c->spawn_radius * q);
  int64_t dmin_int = (int64_t)floor(c->spawn_min * q);
  for (int n = 0; n < n_ent; ++n) {
    int64_t cx = 0, cy = 0; /* last candidate inside the disk (origin if none) */
    for (int t = 0; t < c->spawn_tries; ++t) {
      uint32_t x[4];
      draw(c->seed, (uint32_t)(c->env0 + e), (uint32_t)(n * 64 + t), g, OC_TAG_SPAWN, x);
      int64_t ux = (int64_t)(x[0] >> 8) - 8388608;
      int64_t uy = (int64_t)(x[1] >> 8) - 8388608;
      if (ux * ux + uy * uy > r_int * r_int) continue;
      cx = ux;
      cy = uy;
      int ok = 1;
      for (int m = 0; m < n && ok; ++m) {
        int64_t dx = cx - X[m], dy = cy - Y[m];
        if (dx * dx + dy * dy < dmin_int * dmin_int) ok = 0;
      }
      if (ok) break;
    }
    X[n] = cx;
    Y[n] = cy;
    ex[n] = (double)cx / q;
    ey[n] = (double)cy / q;
  }
}

/* Range of target k seen from agent a: 3-D distance, agent at the surface. */
static double true_range(const oc_state* s, int ia, int it) {
  double dx = s->ax[ia] - s->tx[it], dy = s->ay[ia] - s->ty[it], dz = 0.0 - s->tz[it];
  return sqrt(dx * dx + dy * dy + dz * dz);
}

void oc_reset(const oc_config* c, oc_state* s, uint32_t g) {
  const int P = c->n_particles;
  const int AM = c->max_agents;
#pragma omp parallel for schedule(static)
  for (int e = 0; e < c->n_envs; ++e) {
    int A = env_agents(c, e), T = env_targets(c, e);
    int a0 = c->agent_off[e], t0 = c->target_off[e];
    double ex[OC_MAX_AGENTS + OC_MAX_TARGETS], ey[OC_MAX_AGENTS + OC_MAX_TARGETS];
    spawn_env(c, e, g, ex, ey);
    for (int a = 0; a < A; ++a) {
      uint32_t x[4];
      draw(c->seed, (uint32_t)(c->agent0 + a0 + a), 0, g, OC_TAG_AGENT_INIT, x);
      s->ax[a0 + a] = ex[a];
      s->ay[a0 + a] = ey[a];
      s->apsi[a0 + a] = M_PI * (2.0 * u01(x[0]) - 1.0);
      s->rudder[a0 + a] = (c->n_rudder - 1) / 2; /* straight (action_mode 2) */
    }
    for (int k = 0; k < T; ++k) {
      uint32_t x[4];
      draw(c->seed, (uint32_t)(c->target0 + t0 + k), 0, g, OC_TAG_TARGET_INIT, x);
      s->tx[t0 + k] = ex[A + k];
      s->ty[t0 + k] = ey[A + k];
      s->tpsi[t0 + k] = M_PI * (2.0 * u01(x[0]) - 1.0);
      s->tspeed[t0 + k] = c->target_speed_min + (c->target_speed_max - c->target_speed_min) * u01(x[1]);
      s->tz[t0 + k] = c->target_depth_max * u01(x[2]);
    }
    /* At spawn every teammate is within comm range: all poses known. */
    for (int a = 0; a < A; ++a)
      for (int b = 0; b < AM; ++b) {
        int64_t o = (int64_t)(a0 + a) * AM + b;
        s->lpx[o] = b < A ? s->ax[a0 + b] : 0.0;
        s->lpy[o] = b < A ? s->ay[a0 + b] : 0.0;
        s->lpage[o] = 0;
      }
    /* First ping of each filter and particle initialisation around it. */
    for (int j = 0; j < env_filters(c, e); ++j) {
        int a = filter_agent(c, e, j), k = filter_target(c, e, j);
        int f = c->filter_off[e] + j;
        int ia = a0 + a, it = t0 + k;
        double d = true_range(s, ia, it);
        int valid = d <= c->det_radius;
        uint32_t xp[4];
        draw(c->seed, (uint32_t)(c->filter0 + f), 0, g, OC_TAG_RESET_PING, xp);
        double n0, n1;
        normal_pair(xp[0], xp[1], &n0, &n1);
        double r0 = d + c->range_sigma * n0;
        double zk = s->tz[it];
        double horiz = sqrt(fmax(r0 * r0 - zk * zk, 0.0));
        double sx = 0.0, sy = 0.0;
        for (int i = 0; i < P; ++i) {
          uint32_t x[4], y[4];
          draw(c->seed, (uint32_t)(c->filter0 + f), (uint32_t)i, g, OC_TAG_PF_INIT, x);
          draw(c->seed, (uint32_t)(c->filter0 + f), (uint32_t)i, g, OC_TAG_PF_INIT2, y);
          double rho, m0, m1;
          if (valid) {
            normal_pair(x[0], x[1], &m0, &m1);
            rho = horiz + c->range_sigma * m0;
          } else {
            rho = c->det_radius * sqrt(u01(x[0]));
          }
          double phi = 2.0 * M_PI * u01(x[2]);
          double spd = c->pf_vcap * u01(x[3]);
          double chi = 2.0 * M_PI * u01(y[0]);
          int64_t o = (int64_t)f * P + i;
          s->px[o] = s->ax[ia] + rho * cos(phi);
          s->py[o] = s->ay[ia] + rho * sin(phi);
          s->pvx[o] = spd * cos(chi);
          s->pvy[o] = spd * sin(chi);
          if (s->pw) s->pw[o] = 0.0; /* equal weights */
          sx += s->px[o];
          sy += s->py[o];
        }
        s->estx[f] = sx / P;
        s->esty[f] = sy / P;
        s->prev_estx[f] = s->prev2_estx[f] = s->estx[f];
        s->prev_esty[f] = s->prev2_esty[f] = s->esty[f];
        s->velx[f] = s->vely[f] = 0.0;
        s->ring_head[f] = 0;
        s->ring_count[f] = 0;
        for (int j = 0; j < OC_RING * 4; ++j) s->ring[(int64_t)f * OC_RING * 4 + j] = 0.0;
      }
  }
  s->step = g;
  s->t_ep = 0;
}

/* ------------------------------------------------------------------------ */
/* Actions                                                                  */
/* ------------------------------------------------------------------------ */
/* Uniform random action index (config 1 style exploration). */
void oc_random_actions(const oc_config* c, uint32_t g, int32_t n_agents, int32_t* act) {
  for (int i = 0; i < n_agents; ++i) {
    uint32_t x[4];
    draw(c->seed, (uint32_t)(c->agent0 + i), 0, g, OC_TAG_ACTION, x);
    act[i] = (int32_t)(((uint64_t)x[0] * (uint64_t)c->n_actions) >> 32);
  }
}

/* Sampling from the categorical policy output by the Gumbel-max rule:
 * argmax_j (logit_j - log(-log u_j)), first index on ties. */
void oc_gumbel_actions(uint64_t seed, uint32_t g, int32_t agent0, int32_t n_agents, int32_t n_act,
                       const double* logits, int32_t* act, double* gumbel_out) {
  for (int i = 0; i < n_agents; ++i) {
    double best = -INFINITY;
    int32_t arg = 0;
    for (int j = 0; j < n_act; ++j) {
      uint32_t x[4];
      draw(seed, (uint32_t)(agent0 + i), (uint32_t)(j / 4), g, OC_TAG_GUMBEL, x);
      double gj = -log(-log(u01_mid(x[j % 4])));
      if (gumbel_out) gumbel_out[(int64_t)i * n_act + j] = gj;
      double v = logits[(int64_t)i * n_act + j] + gj;
      if (v > best) { best = v; arg = j; }
    }
    act[i] = arg;
  }
}

/* ------------------------------------------------------------------------ */
/* Agent kinematics (Sec. III-A.3): psi' = wrap(psi + theta(gamma) + noise), */
/* p' = p + v dt (cos psi', sin psi').                                      */
/* ------------------------------------------------------------------------ */
void oc_move_agents(const oc_config* c, oc_state* s, const int32_t* act, uint32_t g) {
  int NA = c->agent_off[c->n_envs];
  for (int i = 0; i < NA; ++i) {
    uint32_t x[4];
    draw(c->seed, (uint32_t)(c->agent0 + i), 0, g, OC_TAG_AGENT_NOISE, x);
    double n0, n1;
    normal_pair(x[0], x[1], &n0, &n1);
    int32_t ang = act[i];
    if (c->action_mode == 2) { /* down / keep / up, clamped at the ends */
      ang = s->rudder[i] + act[i] - 1;
      if (ang < 0) ang = 0;
      if (ang > c->n_rudder - 1) ang = c->n_rudder - 1;
      s->rudder[i] = ang;
    }
    double psi = wrap_angle(s->apsi[i] + action_dpsi(c, ang) + c->heading_noise * n0);
    s->apsi[i] = psi;
    s->ax[i] += c->agent_speed * c->dt * cos(psi);
    s->ay[i] += c->agent_speed * c->dt * sin(psi);
  }
}

/* Target motion: model 0 redraws the heading uniformly every step (an
 * erratic random walk); model 1 lets the heading drift by a Gaussian
 * increment (readings C12).  Speed is the per-target speed drawn at reset. */
void oc_move_targets(const oc_config* c, oc_state* s, uint32_t g) {
  int NT = c->target_off[c->n_envs];
  for (int j = 0; j < NT; ++j) {
    uint32_t x[4];
    draw(c->seed, (uint32_t)(c->target0 + j), 0, g, OC_TAG_TARGET_MOVE, x);
    double psi;
    if (c->target_model == 0) {
      psi = wrap_angle(2.0 * M_PI * u01(x[0]));
    } else {
      double n0, n1;
      normal_pair(x[0], x[1], &n0, &n1);
      psi = wrap_angle(s->tpsi[j] + c->target_drift_sigma * n0);
    }
    s->tpsi[j] = psi;
    s->tx[j] += s->tspeed[j] * c->dt * cos(psi);
    s->ty[j] += s->tspeed[j] * c->dt * sin(psi);
  }
}

/* Range-only acoustic pings (Sec. III-A.2; detection limit from the "Why is
 * UTracking difficult" paragraph): a target is heard iff its 3-D distance is
 * within det_radius; the heard range carries Gaussian noise (reading C3). */
void oc_pings(const oc_config* c, const oc_state* s, uint32_t g, double* range, int32_t* valid) {
  /* range, valid: [pairs] */
  for (int e = 0; e < c->n_envs; ++e) {
    int A = env_agents(c, e), T = env_targets(c, e);
    for (int a = 0; a < A; ++a)
      for (int k = 0; k < T; ++k) {
        int q = pair_index(c, e, a, k);
        double d = true_range(s, c->agent_off[e] + a, c->target_off[e] + k);
        uint32_t x[4];
        draw(c->seed, pair_key(c, q), 0, g, OC_TAG_PING, x);
        double n0, n1;
        normal_pair(x[0], x[1], &n0, &n1);
        valid[q] = d <= c->det_radius;
        range[q] = valid[q] ? d + c->range_sigma * n0 : 0.0;
      }
  }
}

/* Communication (Sec. III-A.2): at the end of the step each agent
 * broadcasts its location and observations; agent a receives agent b iff
 * they are within comm_radius and the message is not dropped.  Each
 * filter (a,k) then holds the measurement list of every received agent that
 * heard target k, senders in increasing index. */
void oc_comms(const oc_config* c, oc_state* s, uint32_t g, const double* range, const int32_t* valid,
              int32_t* recv, double* meas, int32_t* meas_n) {
  const int AM = c->max_agents;
  for (int e = 0; e < c->n_envs; ++e) {
    int A = env_agents(c, e), T = env_targets(c, e), a0 = c->agent_off[e];
    for (int a = 0; a < A; ++a) {
      int ia = a0 + a;
      for (int b = 0; b < AM; ++b) {
        int r = 0;
        if (b < A) {
          int ib = a0 + b;
          if (b == a) {
            r = 1;
          } else {
            double dx = s->ax[ia] - s->ax[ib], dy = s->ay[ia] - s->ay[ib];
            uint32_t x[4];
            draw(c->seed, (uint32_t)(c->agent0 + ia), (uint32_t)b, g, OC_TAG_COMM, x);
            r = sqrt(dx * dx + dy * dy) <= c->comm_radius && !(u01(x[0]) < c->comm_drop);
          }
          if (b != a) {
            int64_t o = (int64_t)ia * AM + b;
            if (r) {
              s->lpx[o] = s->ax[ib];
              s->lpy[o] = s->ay[ib];
              s->lpage[o] = 0;
            } else {
              s->lpage[o] += 1;
            }
          }
        }
        recv[(int64_t)ia * AM + b] = r;
      }
      if (c->shared_filter) continue;
      for (int k = 0; k < T; ++k) {
        int f = filter_index(c, e, a, k);
        int n = 0;
        for (int b = 0; b < A; ++b) {
          int qb = pair_index(c, e, b, k);
          if (recv[(int64_t)ia * AM + b] && valid[qb]) {
            double* m = meas + ((int64_t)f * AM + n) * 4;
            m[0] = s->ax[a0 + b];
            m[1] = s->ay[a0 + b];
            m[2] = 0.0;
            m[3] = range[qb];
            n++;
          }
        }
        meas_n[f] = n;
      }
    }
    /* a shared filter (C22) hears every agent of the env that heard its target */
    if (c->shared_filter)
      for (int k = 0; k < T; ++k) {
        int f = c->filter_off[e] + k;
        int n = 0;
        for (int b = 0; b < A; ++b) {
          int qb = pair_index(c, e, b, k);
          if (valid[qb]) {
            double* m = meas + ((int64_t)f * AM + n) * 4;
            m[0] = s->ax[a0 + b];
            m[1] = s->ay[a0 + b];
            m[2] = 0.0;
            m[3] = range[qb];
            n++;
          }
        }
        meas_n[f] = n;
      }
  }
}

/* ------------------------------------------------------------------------ */
/* Systematic resampling with an exact integer CDF (readings C4, C5).        */
/* wmax[i] = exp(l_i - max l) in [0, 1]; q_i = floor(wmax_i 2^38);           */
/* Q_i = sum_{l<=i} q_l; W = Q_{P-1}; offset U0 = floor(u64 W / 2^64);       */
/* idx_j = min{ i : P Q_i > j W + U0 }.  This is systematic resampling with  */
/* u_j = (j + U0/W) / P on the normalised CDF C_i = Q_i / W.                 */
/* ------------------------------------------------------------------------ */
void oc_systematic_resample(int32_t P, const double* wmax, uint64_t u64, int32_t* idx) {
  int64_t* Q = (int64_t*)malloc(sizeof(int64_t) * (size_t)P);
  int64_t acc = 0;
  for (int i = 0; i < P; ++i) {
    acc += (int64_t)floor(wmax[i] * 274877906944.0); /* 2^38 */
    Q[i] = acc;
  }
  int64_t W = Q[P - 1];
  int64_t U0 = (int64_t)(((unsigned __int128)u64 * (unsigned __int128)(uint64_t)W) >> 64);
  int i = 0;
  for (int j = 0; j < P; ++j) {
    int64_t thr = (int64_t)j * W + U0;
    while ((int64_t)P * Q[i] <= thr) ++i;
    idx[j] = i;
  }
  free(Q);
}

/* ------------------------------------------------------------------------ */
/* Particle filter update of every (env, agent, target) tracker (Sec. II-A,  */
/* Sec. III-A.2: one tracker per agent per target).  State (x, y, vx, vy).   */
/* Predict: v += sigma_a N(0, I); |v| capped at v_cap; p += dt v (C2).       */
/* Weight: Gaussian range likelihood over the received measurements (C3),    */
/* normalised.  Estimate: weighted mean before resampling (C6).  Resample:   */
/* systematic, every step with at least one measurement (C4).                */
/* ------------------------------------------------------------------------ */
void oc_pf_update(const oc_config* c, oc_state* s, uint32_t g, const double* meas, const int32_t* meas_n,
                  oc_step_out* o) {
  const int P = c->n_particles;
  const int AM = c->max_agents;
  int F = c->filter_off[c->n_envs];
#pragma omp parallel for schedule(dynamic, 4)
  for (int f = 0; f < F; ++f) {
    /* Which env does filter f belong to?  (binary search on the offsets) */
    int lo = 0, hi = c->n_envs - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) / 2;
      if (c->filter_off[mid] <= f) lo = mid; else hi = mid - 1;
    }
    int e = lo;
    int T = env_targets(c, e);
    int k = (f - c->filter_off[e]) % T;
    int it = c->target_off[e] + k;
    double* x = s->px + (int64_t)f * P;
    double* y = s->py + (int64_t)f * P;
    double* vx = s->pvx + (int64_t)f * P;
    double* vy = s->pvy + (int64_t)f * P;
    double* l = (double*)malloc(sizeof(double) * P * 6);
    double* w = l + P;
    double* ox = l + 2 * P;
    double* oy = l + 3 * P;
    double* ovx = l + 4 * P;
    double* ovy = l + 5 * P;
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * P);
    /* predict */
    for (int i = 0; i < P; ++i) {
      uint32_t r[4];
      draw(c->seed, (uint32_t)(c->filter0 + f), (uint32_t)(i / 2), g, OC_TAG_PF_PREDICT, r);
      double n0, n1;
      if (i % 2 == 0) normal_pair(r[0], r[1], &n0, &n1);
      else normal_pair(r[2], r[3], &n0, &n1);
      vx[i] += c->pf_accel_sigma * n0;
      vy[i] += c->pf_accel_sigma * n1;
      double sp = sqrt(vx[i] * vx[i] + vy[i] * vy[i]);
      if (sp > c->pf_vcap) {
        vx[i] *= c->pf_vcap / sp;
        vy[i] *= c->pf_vcap / sp;
      }
      x[i] += c->dt * vx[i];
      y[i] += c->dt * vy[i];
    }
    int nm = meas_n[f];
    const double* m = meas + (int64_t)f * AM * 4;
    /* weight */
    double lmax = -INFINITY;
    for (int i = 0; i < P; ++i) {
      double acc = 0.0;
      for (int j = 0; j < nm; ++j) {
        double dx = x[i] - m[j * 4 + 0], dy = y[i] - m[j * 4 + 1], dz = s->tz[it] - m[j * 4 + 2];
        double res = m[j * 4 + 3] - sqrt(dx * dx + dy * dy + dz * dz);
        acc += res * res;
      }
      /* log-likelihood, plus the carried log-weight when resampling is
       * triggered by the effective sample size (reading C23) */
      l[i] = (c->pf_ess_num > 0 ? s->pw[(int64_t)f * P + i] : 0.0) - acc / (2.0 * c->range_sigma * c->range_sigma);
      if (l[i] > lmax) lmax = l[i];
    }
    double W = 0.0;
    for (int i = 0; i < P; ++i) {
      w[i] = exp(l[i] - lmax);
      W += w[i];
    }
    /* resample every step with a measurement, or (C23) only when
     * 16 (sum r)^2 < k P sum r^2 with r = floor(w 2^38) >> 23; the carried
     * log-weights become 0 after a resample, l - max l otherwise */
    int resample = nm > 0;
    if (c->pf_ess_num > 0) {
      uint64_t s1 = 0, s2 = 0;
      for (int i = 0; i < P; ++i) {
        uint64_t r = (uint64_t)(int64_t)floor(w[i] * 274877906944.0) >> 23;
        s1 += r;
        s2 += r * r;
      }
      resample = resample && 16u * s1 * s1 < (uint64_t)c->pf_ess_num * (uint64_t)P * s2;
      for (int i = 0; i < P; ++i) s->pw[(int64_t)f * P + i] = resample ? 0.0 : l[i] - lmax;
    }
    /* estimate (weighted mean; uniform weights when nothing was heard) */
    double ex = 0.0, ey = 0.0;
    for (int i = 0; i < P; ++i) {
      ex += (w[i] / W) * x[i];
      ey += (w[i] / W) * y[i];
    }
    /* smoothed motion of the estimate (reading C18): v <- 0.85 v + 0.15 (e1 - e2)
     * with e1 the estimate before this update and e2 the one before that */
    s->velx[f] = OC_VEL_KEEP * s->velx[f] + (1.0 - OC_VEL_KEEP) * (s->estx[f] - s->prev_estx[f]);
    s->vely[f] = OC_VEL_KEEP * s->vely[f] + (1.0 - OC_VEL_KEEP) * (s->esty[f] - s->prev_esty[f]);
    s->prev2_estx[f] = s->prev_estx[f];
    s->prev2_esty[f] = s->prev_esty[f];
    s->prev_estx[f] = s->estx[f];
    s->prev_esty[f] = s->esty[f];
    s->estx[f] = ex;
    s->esty[f] = ey;
    double dxe = ex - s->tx[it], dye = ey - s->ty[it];
    if (o && o->err) o->err[f] = sqrt(dxe * dxe + dye * dye);
    if (o && o->pred_px)
      for (int i = 0; i < P; ++i) {
        int64_t q = (int64_t)f * P + i;
        o->pred_px[q] = x[i];
        o->pred_py[q] = y[i];
        o->pred_pvx[q] = vx[i];
        o->pred_pvy[q] = vy[i];
      }
    if (o && o->weight)
      for (int i = 0; i < P; ++i) o->weight[(int64_t)f * P + i] = w[i] / W;
    if (o && o->wmax)
      for (int i = 0; i < P; ++i) o->wmax[(int64_t)f * P + i] = w[i];
    /* resample */
    if (resample) {
      uint32_t r[4];
      draw(c->seed, (uint32_t)(c->filter0 + f), 0, g, OC_TAG_RESAMPLE, r);
      uint64_t u64 = (uint64_t)r[0] | ((uint64_t)r[1] << 32);
      oc_systematic_resample(P, w, u64, idx);
      for (int j = 0; j < P; ++j) {
        ox[j] = x[idx[j]];
        oy[j] = y[idx[j]];
        ovx[j] = vx[idx[j]];
        ovy[j] = vy[idx[j]];
      }
      memcpy(x, ox, sizeof(double) * P);
      memcpy(y, oy, sizeof(double) * P);
      memcpy(vx, ovx, sizeof(double) * P);
      memcpy(vy, ovy, sizeof(double) * P);
    } else {
      for (int j = 0; j < P; ++j) idx[j] = j;
    }
    if (o && o->idx)
      for (int j = 0; j < P; ++j) o->idx[(int64_t)f * P + j] = idx[j];
    free(idx);
    free(l);
  }
}

/* ------------------------------------------------------------------------ */
/* Observation tokens (Sec. III-A.2 "Observation Space", Fig. 3): per agent  */
/* one 8-feature vector per entity: relative 3-D offset / S, one-hot        */
/* {self, agent, target}, "missing" (teammate not heard this step), age of  */
/* the teammate pose / 16 (capped at 1).  Teammates use the last received   */
/* pose, targets the agent's own tracker estimate.  Order: self, teammates  */
/* in index order, targets in index order; the remaining slots are zero     */
/* padding (masked by the entity count A_e + T_e).                          */
/* ------------------------------------------------------------------------ */
void oc_obs(const oc_config* c, const oc_state* s, double* tokens) {
  const int AM = c->max_agents, NS = c->max_agents + c->max_targets;
  const double S = c->feature_scale;
  for (int e = 0; e < c->n_envs; ++e) {
    int A = env_agents(c, e), T = env_targets(c, e), a0 = c->agent_off[e];
    for (int a = 0; a < A; ++a) {
      int ia = a0 + a;
      double* tk = tokens + (int64_t)ia * NS * OC_TOKEN;
      for (int j = 0; j < NS * OC_TOKEN; ++j) tk[j] = 0.0;
      tk[3] = 1.0; /* slot 0: self */
      int slot = 1;
      for (int b = 0; b < A; ++b) {
        if (b == a) continue;
        int64_t o = (int64_t)ia * AM + b;
        double* t = tk + slot * OC_TOKEN;
        t[0] = (s->lpx[o] - s->ax[ia]) / S;
        t[1] = (s->lpy[o] - s->ay[ia]) / S;
        t[2] = 0.0;
        t[4] = 1.0;
        t[6] = s->lpage[o] > 0 ? 1.0 : 0.0;
        t[7] = (s->lpage[o] < 16 ? (double)s->lpage[o] : 16.0) / 16.0;
        slot++;
      }
      for (int k = 0; k < T; ++k) {
        int f = filter_index(c, e, a, k);
        double* t = tk + slot * OC_TOKEN;
        t[0] = (s->estx[f] - s->ax[ia]) / S;
        t[1] = (s->esty[f] - s->ay[ia]) / S;
        t[2] = s->tz[c->target_off[e] + k] / S;
        t[5] = 1.0;
        slot++;
      }
    }
  }
}

/* Tracking reward Eq. (1) for one error value. */
double oc_tracking_reward(double err, double eps_min, double eps_max) {
  if (err < eps_min) return 1.0;
  if (err > eps_max) return 0.0;
  double t = (err - eps_min) / (eps_max - eps_min);
  if (t >= 1.0) return 0.0; /* limit of exp(-2t/(1-t)) as t -> 1 */
  return exp(-2.0 * t / (1.0 - t));
}

/* Reward (Sec. III-A.2 "Reward Function"): per-target Eq. (1) on the
 * agent-averaged tracking error (reading C14) or Eq. (2) follow indicator on
 * the nearest-agent distance; averaged over targets; -1 if any two agents
 * are closer than d_safe. */
void oc_reward(const oc_config* c, const oc_state* s, const double* err, double* reward, int32_t* crash) {
  for (int e = 0; e < c->n_envs; ++e) {
    int A = env_agents(c, e), T = env_targets(c, e), a0 = c->agent_off[e], t0 = c->target_off[e];
    double r = 0.0;
    for (int k = 0; k < T; ++k) {
      if (c->reward_type == 0) {
        double ek = 0.0;
        if (c->shared_filter) { /* every agent's error is the shared filter's */
          ek = err[filter_index(c, e, 0, k)];
        } else {
          for (int a = 0; a < A; ++a) ek += err[filter_index(c, e, a, k)];
          ek /= A;
        }
        r += oc_tracking_reward(ek, c->eps_min, c->eps_max);
      } else {
        double dk = INFINITY;
        for (int a = 0; a < A; ++a) {
          double dx = s->ax[a0 + a] - s->tx[t0 + k], dy = s->ay[a0 + a] - s->ty[t0 + k];
          double d = sqrt(dx * dx + dy * dy);
          if (d < dk) dk = d;
        }
        r += dk <= c->follow_dmin ? 1.0 : 0.0;
      }
    }
    r /= T;
    int cr = 0;
    for (int a = 0; a < A; ++a)
      for (int b = a + 1; b < A; ++b) {
        double dx = s->ax[a0 + a] - s->ax[a0 + b], dy = s->ay[a0 + a] - s->ay[a0 + b];
        if (sqrt(dx * dx + dy * dy) < c->d_safe) cr = 1;
      }
    if (cr) r = -1.0;
    reward[e] = r;
    if (crash) crash[e] = cr;
  }
}

/* ------------------------------------------------------------------------ */
/* Learned range-only estimator inputs (reading C18): append this step's     */
/* measurement list of filter (a,k) to its 16-entry ring.  After the step,   */
/* the features of the filter's update are, in the local frame of the       */
/* estimate e1 it updated (units of L): 16 slots newest first x             */
/* [(q - e1)/L, (r - |q - e1|_3D)/L, (g - g_m)/16, valid], then the         */
/* estimate's last motion (e1 - e2)/L, zero padded to 96; the label is the  */
/* correction (x_true - e1)/L.                                              */
/* ------------------------------------------------------------------------ */
void oc_ring_append(const oc_config* c, oc_state* s, uint32_t g, const double* meas, const int32_t* meas_n) {
  const int AM = c->max_agents;
  int F = c->filter_off[c->n_envs];
  for (int f = 0; f < F; ++f) {
    for (int j = 0; j < meas_n[f]; ++j) {
      const double* m = meas + ((int64_t)f * AM + j) * 4;
      double* slot = s->ring + ((int64_t)f * OC_RING + s->ring_head[f]) * 4;
      slot[0] = m[0];
      slot[1] = m[1];
      slot[2] = m[3];
      slot[3] = (double)g;
      s->ring_head[f] = (s->ring_head[f] + 1) % OC_RING;
      if (s->ring_count[f] < OC_RING) s->ring_count[f]++;
    }
  }
}

void oc_est_features(const oc_config* c, const oc_state* s, uint32_t g, double* feat, double* label) {
  const double L = c->est_scale;
  for (int e = 0; e < c->n_envs; ++e) {
    for (int j = 0; j < env_filters(c, e); ++j) {
        int k = filter_target(c, e, j);
        int f = c->filter_off[e] + j;
        int it = c->target_off[e] + k;
        double e1x = s->prev_estx[f], e1y = s->prev_esty[f];
        double* x = feat + (int64_t)f * OC_FEAT;
        for (int j = 0; j < OC_FEAT; ++j) x[j] = 0.0;
        for (int sl = 0; sl < s->ring_count[f]; ++sl) {
          int pos = ((s->ring_head[f] - 1 - sl) % OC_RING + OC_RING) % OC_RING;
          const double* r = s->ring + ((int64_t)f * OC_RING + pos) * 4;
          double dx = r[0] - e1x, dy = r[1] - e1y, dz = s->tz[it];
          double rho = sqrt(dx * dx + dy * dy + dz * dz);
          x[sl * 5 + 0] = dx / L;
          x[sl * 5 + 1] = dy / L;
          x[sl * 5 + 2] = (r[2] - rho) / L;
          x[sl * 5 + 3] = ((double)g - r[3]) / 16.0;
          x[sl * 5 + 4] = 1.0;
        }
        x[5 * OC_RING + 0] = (e1x - s->prev2_estx[f]) / L;
        x[5 * OC_RING + 1] = (e1y - s->prev2_esty[f]) / L;
        x[5 * OC_RING + 2] = s->velx[f] / L;
        x[5 * OC_RING + 3] = s->vely[f] / L;
        if (label) {
          label[(int64_t)f * 2 + 0] = (s->tx[it] - e1x) / L;
          label[(int64_t)f * 2 + 1] = (s->ty[it] - e1y) / L;
        }
      }
  }
}

/* ------------------------------------------------------------------------ */
/* One environment step in the order of reading C7: move agents, move        */
/* targets, ping, communicate, update trackers, observe, reward.             */
/* ------------------------------------------------------------------------ */
/* ------------------------------------------------------------------------ */
/* Learned form of the tracker update (readings C18): the estimator network  */
/* (oc_mlp_forward, utrack_oracle_nn.c) moves each filter's estimate e1 by    */
/* L * clamp(out, +-3) on a step with a fresh ping.  Without one, mode 1      */
/* holds e1, mode 2 applies the network all the same, mode 3 coasts by the    */
/* smoothed motion v.  The history (e2 <- e1 <- estimate, v) is advanced      */
/* first, so the features are those of oc_est_features for this step.        */
/* ------------------------------------------------------------------------ */
void oc_mlp_forward(int32_t B, const double* params, const double* X, double* out, double* pre);

static void oc_learned_update(const oc_config* c, oc_state* s, uint32_t g, const double* mlp, int32_t mode,
                              double* err) {
  const int F = c->filter_off[c->n_envs];
  const double L = c->est_scale;
  for (int f = 0; f < F; ++f) {
    s->velx[f] = OC_VEL_KEEP * s->velx[f] + (1.0 - OC_VEL_KEEP) * (s->estx[f] - s->prev_estx[f]);
    s->vely[f] = OC_VEL_KEEP * s->vely[f] + (1.0 - OC_VEL_KEEP) * (s->esty[f] - s->prev_esty[f]);
    s->prev2_estx[f] = s->prev_estx[f];
    s->prev2_esty[f] = s->prev_esty[f];
    s->prev_estx[f] = s->estx[f];
    s->prev_esty[f] = s->esty[f];
  }
  double* feat = (double*)malloc(sizeof(double) * (size_t)F * OC_FEAT);
  double* out = (double*)malloc(sizeof(double) * (size_t)F * 2);
  oc_est_features(c, s, g, feat, NULL);
  oc_mlp_forward(F, mlp, feat, out, NULL);
  for (int e = 0; e < c->n_envs; ++e) {
    for (int j = 0; j < env_filters(c, e); ++j) {
        int k = filter_target(c, e, j);
        int f = c->filter_off[e] + j;
        int it = c->target_off[e] + k;
        const double* x = feat + (int64_t)f * OC_FEAT;
        int fresh = x[3] == 0.0 && x[4] == 1.0;
        double lim = (fresh || mode == 2) ? 3.0 : 0.0;
        double c0 = fmin(fmax(out[2 * (int64_t)f], -lim), lim);
        double c1 = fmin(fmax(out[2 * (int64_t)f + 1], -lim), lim);
        if (!fresh && mode == 3) {
          c0 = fmin(fmax(x[5 * OC_RING + 2], -3.0), 3.0);
          c1 = fmin(fmax(x[5 * OC_RING + 3], -3.0), 3.0);
        }
        s->estx[f] = s->prev_estx[f] + L * c0;
        s->esty[f] = s->prev_esty[f] + L * c1;
        double dx = s->estx[f] - s->tx[it], dy = s->esty[f] - s->ty[it];
        err[f] = sqrt(dx * dx + dy * dy);
      }
  }
  free(feat);
  free(out);
}

/* ------------------------------------------------------------------------ */
/* Least-squares trilateration tracker (Sec. II-A; Sec. III-A.2 names LS and  */
/* PF as the two tracking models), reading C21.  The pings in the filter's    */
/* ring, horizontal ranges rho = sqrt(max(r^2 - dz^2, 0)) with the target     */
/* depth known, the target static over the window: |x - q|^2 = rho^2 gives    */
/* 2 q.x = |x|^2 + a, a = |q|^2 - rho^2; subtracting the mean over the pings  */
/* leaves the linear system 2 (q_m - qbar).x = a_m - abar, solved in the      */
/* least-squares sense by the 2 x 2 normal equations.  Positions relative to  */
/* the previous estimate e1.  Fewer than 3 pings, or det A <= 1e-3 (tr A)^2,  */
/* hold e1.                                                                   */
/* ------------------------------------------------------------------------ */
#define OC_LS_MIN_DET_RATIO 1e-3

void oc_ls_update(const oc_config* c, oc_state* s, double* err) {
  for (int e = 0; e < c->n_envs; ++e) {
    for (int j = 0; j < env_filters(c, e); ++j) {
        int k = filter_target(c, e, j);
        int f = c->filter_off[e] + j;
        int it = c->target_off[e] + k;
        double e1x = s->estx[f], e1y = s->esty[f], dz = s->tz[it];
        int n = s->ring_count[f];
        double qx[OC_RING], qy[OC_RING], av[OC_RING], mx = 0.0, my = 0.0, ma = 0.0;
        for (int sl = 0; sl < n; ++sl) {
          int pos = ((s->ring_head[f] - 1 - sl) % OC_RING + OC_RING) % OC_RING;
          const double* r = s->ring + ((int64_t)f * OC_RING + pos) * 4;
          double rho2 = fmax(r[2] * r[2] - dz * dz, 0.0);
          qx[sl] = r[0] - e1x;
          qy[sl] = r[1] - e1y;
          av[sl] = qx[sl] * qx[sl] + qy[sl] * qy[sl] - rho2;
          mx += qx[sl];
          my += qy[sl];
          ma += av[sl];
        }
        double ex = e1x, ey = e1y;
        if (n >= 3) {
          mx /= n;
          my /= n;
          ma /= n;
          double a00 = 0.0, a01 = 0.0, a11 = 0.0, b0 = 0.0, b1 = 0.0;
          for (int sl = 0; sl < n; ++sl) {
            double dx = qx[sl] - mx, dy = qy[sl] - my, da = av[sl] - ma;
            a00 += dx * dx;
            a01 += dx * dy;
            a11 += dy * dy;
            b0 += 0.5 * dx * da;
            b1 += 0.5 * dy * da;
          }
          double det = a00 * a11 - a01 * a01, tr = a00 + a11;
          if (det > OC_LS_MIN_DET_RATIO * tr * tr) {
            ex = e1x + (a11 * b0 - a01 * b1) / det;
            ey = e1y + (a00 * b1 - a01 * b0) / det;
          }
        }
        s->velx[f] = OC_VEL_KEEP * s->velx[f] + (1.0 - OC_VEL_KEEP) * (e1x - s->prev_estx[f]);
        s->vely[f] = OC_VEL_KEEP * s->vely[f] + (1.0 - OC_VEL_KEEP) * (e1y - s->prev_esty[f]);
        s->prev2_estx[f] = s->prev_estx[f];
        s->prev2_esty[f] = s->prev_esty[f];
        s->prev_estx[f] = e1x;
        s->prev_esty[f] = e1y;
        s->estx[f] = ex;
        s->esty[f] = ey;
        double dxe = ex - s->tx[it], dye = ey - s->ty[it];
        err[f] = sqrt(dxe * dxe + dye * dye);
      }
  }
}

static void step_impl(const oc_config* c, oc_state* s, const int32_t* act, oc_step_out* o, const double* mlp,
                      int32_t mode) {
  int F = c->filter_off[c->n_envs];
  int NPAIR = c->pair_off[c->n_envs];
  int NA = c->agent_off[c->n_envs];
  int AM = c->max_agents;
  uint32_t g = s->step + 1;
  double* range = (double*)malloc(sizeof(double) * NPAIR);
  int32_t* valid = (int32_t*)malloc(sizeof(int32_t) * NPAIR);
  int32_t* recv = (int32_t*)malloc(sizeof(int32_t) * (size_t)NA * AM);
  double* meas = (double*)malloc(sizeof(double) * (size_t)F * AM * 4);
  int32_t* meas_n = (int32_t*)malloc(sizeof(int32_t) * F);
  double* err = (double*)malloc(sizeof(double) * F);
  oc_move_agents(c, s, act, g);
  oc_move_targets(c, s, g);
  oc_pings(c, s, g, range, valid);
  oc_comms(c, s, g, range, valid, recv, meas, meas_n);
  oc_ring_append(c, s, g, meas, meas_n);
  oc_step_out local = {0};
  if (o) local = *o;
  local.err = err;
  if (mode == 4)
    oc_ls_update(c, s, err);
  else if (mlp)
    oc_learned_update(c, s, g, mlp, mode, err);
  else
    oc_pf_update(c, s, g, meas, meas_n, &local);
  if (o && o->tokens) oc_obs(c, s, o->tokens);
  if (o && o->reward) oc_reward(c, s, err, o->reward, o->crash);
  if (o && o->range) memcpy(o->range, range, sizeof(double) * NPAIR);
  if (o && o->valid) memcpy(o->valid, valid, sizeof(int32_t) * NPAIR);
  if (o && o->recv) memcpy(o->recv, recv, sizeof(int32_t) * (size_t)NA * AM);
  if (o && o->meas) memcpy(o->meas, meas, sizeof(double) * (size_t)F * AM * 4);
  if (o && o->meas_n) memcpy(o->meas_n, meas_n, sizeof(int32_t) * F);
  if (o && o->err) memcpy(o->err, err, sizeof(double) * F);
  s->step = g;
  s->t_ep += 1;
  free(range); free(valid); free(recv); free(meas); free(meas_n); free(err);
}

void oc_step(const oc_config* c, oc_state* s, const int32_t* act, oc_step_out* o) { step_impl(c, s, act, o, NULL, 0); }

/* The same step with the learned tracker (mode 1, 2 or 3 as above) or, with
 * mode 4, the least-squares tracker (mlp unused). */
void oc_step_learned(const oc_config* c, oc_state* s, const int32_t* act, const double* mlp, int32_t mode,
                     oc_step_out* o) {
  step_impl(c, s, act, o, mlp, mode);
}
