/*
 * FP64 CPU oracle, TransfMAPPO training: the loss gradients of the
 * transformer actor and critic, generalized advantage estimation and the
 * critic's global-state tokens.
 *
 * TEST INFRASTRUCTURE ONLY (see utrack_oracle.c).  Shares nothing with the
 * CUDA path.  Every product and sum is in double.
 *
 * Method (Sec. II-B, Sec. III-B.1, Fig. 3):
 *  - MAPPO: each actor is trained with PPO's clipped surrogate objective and
 *    a single centralized critic estimates V(S) from the global state;
 *    CTDE, the critic is used in training only.
 *  - TransformerAgent (actor) and TransformerCritic share one architecture:
 *    entity tokens embedded as graph vertices, an extra recurrent embedding
 *    processed jointly, self-attention blocks, LayerNorm throughout, an MLP
 *    head on the transformed recurrent embedding (action logits for the
 *    actor, the value for the critic).
 *  - The critic's tokens are the true position, velocity and heading of every
 *    agent and target (the global state of Sec. III-A, observation space).
 * Readings (the paper gives no formulas for these parts):
 *  - architecture as the agent's forward (pre-LN, FFN 4d with erf-GELU,
 *    LayerNorm epsilon 1e-5, final LayerNorm + linear head on token 0);
 *  - PPO (Schulman et al. 2017, Eq. 7, with the entropy bonus of Eq. 9):
 *    per sample L = -min(r A, clip(r, 1-eps, 1+eps) A) - c_ent H(pi),
 *    r = exp(log pi(a) - log pi_old(a)); the batch loss is the mean;
 *  - value loss: the mean of (V - R)^2 over samples (no value clipping);
 *  - the recurrent input of a sample is data (no backpropagation through
 *    time: the gradient stops at the recorded recurrent embedding);
 *  - advantages: GAE (Schulman et al. 2016, Eq. 16) with the sum cut after
 *    the step that ends an episode; returns R = A + V.
 *
 * Pins: gradients against central finite differences, the clipped region's
 * zero gradient, closed forms of GAE (lambda = 0: one-step TD error;
 * lambda = 1: discounted return minus the value), permutation invariance of
 * the critic over entity tokens.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t d, n_layers, n_heads, n_out, n_in;
} oc_tfm_dims;

static double g_gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }
static double g_gelu_grad(double x) {
  return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
}

/* Parameter views in the canonical order of the transformer agent (see
 * oc_policy_param_count); n_out replaces the number of actions. */
typedef struct {
  const double *W_emb, *b_emb;
  const double *ln1_g[8], *ln1_b[8], *Wqkv[8], *bqkv[8], *Wo[8], *bo[8];
  const double *ln2_g[8], *ln2_b[8], *W1[8], *b1[8], *W2[8], *b2[8];
  const double *lnf_g, *lnf_b, *Wh, *bh;
} tfm_view;

int64_t oc_tfm_param_count(const oc_tfm_dims* p) {
  int64_t d = p->d;
  int64_t per_layer = 2 * d + 3 * d * d + 3 * d + d * d + d + 2 * d + 4 * d * d + 4 * d + 4 * d * d + d;
  return d * p->n_in + d + p->n_layers * per_layer + 2 * d + (int64_t)p->n_out * d + p->n_out;
}

/* Offsets of the views inside a flat array (the same split serves the
 * parameters and the gradient). */
static void tfm_offsets(const oc_tfm_dims* p, int64_t* off) {
  const int64_t d = p->d, f = 4 * d;
  int64_t o = 0, k = 0;
  off[k++] = o; o += d * p->n_in;
  off[k++] = o; o += d;
  for (int l = 0; l < p->n_layers; ++l) {
    const int64_t sz[12] = {d, d, 3 * d * d, 3 * d, d * d, d, d, d, f * d, f, d * f, d};
    for (int j = 0; j < 12; ++j) {
      off[k++] = o;
      o += sz[j];
    }
  }
  off[k++] = o; o += d;
  off[k++] = o; o += d;
  off[k++] = o; o += (int64_t)p->n_out * d;
  off[k++] = o;
}

static tfm_view tfm_split(const oc_tfm_dims* p, const double* q) {
  int64_t off[4 + 12 * 8 + 4];
  tfm_offsets(p, off);
  tfm_view v;
  int k = 0;
  v.W_emb = q + off[k++];
  v.b_emb = q + off[k++];
  for (int l = 0; l < p->n_layers; ++l) {
    v.ln1_g[l] = q + off[k++]; v.ln1_b[l] = q + off[k++];
    v.Wqkv[l] = q + off[k++]; v.bqkv[l] = q + off[k++];
    v.Wo[l] = q + off[k++]; v.bo[l] = q + off[k++];
    v.ln2_g[l] = q + off[k++]; v.ln2_b[l] = q + off[k++];
    v.W1[l] = q + off[k++]; v.b1[l] = q + off[k++];
    v.W2[l] = q + off[k++]; v.b2[l] = q + off[k++];
  }
  v.lnf_g = q + off[k++];
  v.lnf_b = q + off[k++];
  v.Wh = q + off[k++];
  v.bh = q + off[k++];
  return v;
}

/* Writable gradient views: the same offsets applied to the gradient array. */
typedef struct {
  double *W_emb, *b_emb;
  double *ln1_g[8], *ln1_b[8], *Wqkv[8], *bqkv[8], *Wo[8], *bo[8];
  double *ln2_g[8], *ln2_b[8], *W1[8], *b1[8], *W2[8], *b2[8];
  double *lnf_g, *lnf_b, *Wh, *bh;
} tfm_gview;

static tfm_gview tfm_gsplit(const oc_tfm_dims* p, double* q) {
  tfm_view c = tfm_split(p, q);
  tfm_gview g;
  g.W_emb = (double*)c.W_emb; g.b_emb = (double*)c.b_emb;
  for (int l = 0; l < p->n_layers; ++l) {
    g.ln1_g[l] = (double*)c.ln1_g[l]; g.ln1_b[l] = (double*)c.ln1_b[l];
    g.Wqkv[l] = (double*)c.Wqkv[l]; g.bqkv[l] = (double*)c.bqkv[l];
    g.Wo[l] = (double*)c.Wo[l]; g.bo[l] = (double*)c.bo[l];
    g.ln2_g[l] = (double*)c.ln2_g[l]; g.ln2_b[l] = (double*)c.ln2_b[l];
    g.W1[l] = (double*)c.W1[l]; g.b1[l] = (double*)c.b1[l];
    g.W2[l] = (double*)c.W2[l]; g.b2[l] = (double*)c.b2[l];
  }
  g.lnf_g = (double*)c.lnf_g; g.lnf_b = (double*)c.lnf_b; g.Wh = (double*)c.Wh; g.bh = (double*)c.bh;
  return g;
}

/* y = W x + b, W [n][k] row-major */
static void mv(int n, int k, const double* W, const double* b, const double* x, double* y) {
  for (int i = 0; i < n; ++i) {
    double acc = b ? b[i] : 0.0;
    for (int j = 0; j < k; ++j) acc += W[(int64_t)i * k + j] * x[j];
    y[i] = acc;
  }
}

/* x += W^T y, W [n][k] */
static void mtv_add(int n, int k, const double* W, const double* y, double* x) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < k; ++j) x[j] += W[(int64_t)i * k + j] * y[i];
}

/* G[n][k] += y x^T (outer product) */
static void outer_add(int n, int k, const double* y, const double* x, double* G) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < k; ++j) G[(int64_t)i * k + j] += y[i] * x[j];
}

/* LayerNorm with the normalised input kept: xh = (x - mean) / sqrt(var + 1e-5) */
static void ln_fwd(int d, const double* x, const double* g, const double* b, double* xh, double* rstd, double* y) {
  double mu = 0.0, var = 0.0;
  for (int i = 0; i < d; ++i) mu += x[i];
  mu /= d;
  for (int i = 0; i < d; ++i) var += (x[i] - mu) * (x[i] - mu);
  var /= d;
  *rstd = 1.0 / sqrt(var + 1e-5);
  for (int i = 0; i < d; ++i) {
    xh[i] = (x[i] - mu) * (*rstd);
    y[i] = xh[i] * g[i] + b[i];
  }
}

/* Backward of y = xh * g + b with xh the normalised x: accumulates dg, db
 * and adds dL/dx to dx. */
static void ln_bwd(int d, const double* xh, double rstd, const double* g, const double* dy, double* dg, double* db,
                   double* dx) {
  double m1 = 0.0, m2 = 0.0;
  for (int i = 0; i < d; ++i) {
    const double dxh = dy[i] * g[i];
    dg[i] += dy[i] * xh[i];
    db[i] += dy[i];
    m1 += dxh;
    m2 += dxh * xh[i];
  }
  m1 /= d;
  m2 /= d;
  for (int i = 0; i < d; ++i) dx[i] += rstd * (dy[i] * g[i] - m1 - xh[i] * m2);
}

/* Activations of one sample kept for the backward pass. */
typedef struct {
  int n;                                  /* tokens: 1 + entities */
  double *X[9];                           /* residual stream entering block l, and X[L] = output */
  double *xh1, *r1, *QKV, *P, *O, *M, *xh2, *r2, *Z, *G;  /* per layer, [L][...] */
  double *xhf, rf, *U;                    /* final LayerNorm on token 0 */
  double *out;                            /* head output [n_out] */
} tfm_cache;

static void* xmalloc(size_t n) { return calloc(n ? n : 1, 1); }

static void cache_alloc(const oc_tfm_dims* p, int n, tfm_cache* c) {
  const int d = p->d, L = p->n_layers, H = p->n_heads;
  c->n = n;
  for (int l = 0; l <= L; ++l) c->X[l] = (double*)xmalloc(sizeof(double) * n * d);
  c->xh1 = (double*)xmalloc(sizeof(double) * L * n * d);
  c->r1 = (double*)xmalloc(sizeof(double) * L * n);
  c->QKV = (double*)xmalloc(sizeof(double) * L * n * 3 * d);
  c->P = (double*)xmalloc(sizeof(double) * L * H * n * n);
  c->O = (double*)xmalloc(sizeof(double) * L * n * d);
  c->M = (double*)xmalloc(sizeof(double) * L * n * d);
  c->xh2 = (double*)xmalloc(sizeof(double) * L * n * d);
  c->r2 = (double*)xmalloc(sizeof(double) * L * n);
  c->Z = (double*)xmalloc(sizeof(double) * L * n * 4 * d);
  c->G = (double*)xmalloc(sizeof(double) * L * n * 4 * d);
  c->xhf = (double*)xmalloc(sizeof(double) * d);
  c->U = (double*)xmalloc(sizeof(double) * d);
  c->out = (double*)xmalloc(sizeof(double) * p->n_out);
}

static void cache_free(const oc_tfm_dims* p, tfm_cache* c) {
  for (int l = 0; l <= p->n_layers; ++l) free(c->X[l]);
  free(c->xh1); free(c->r1); free(c->QKV); free(c->P); free(c->O); free(c->M);
  free(c->xh2); free(c->r2); free(c->Z); free(c->G); free(c->xhf); free(c->U); free(c->out);
}

/* Forward pass of one sample: token 0 is the recurrent embedding h, tokens
 * 1..n-1 the embedded entity vectors tok[0..n-2]. */
static void tfm_fwd(const oc_tfm_dims* p, const tfm_view* v, const double* tok, const double* h, tfm_cache* c) {
  const int d = p->d, H = p->n_heads, dh = p->d / p->n_heads, f = 4 * p->d, n = c->n;
  double* y = (double*)xmalloc(sizeof(double) * (size_t)(f > 3 * d ? f : 3 * d));
  double* s = (double*)xmalloc(sizeof(double) * n);
  for (int j = 0; j < d; ++j) c->X[0][j] = h[j];
  for (int t = 1; t < n; ++t) mv(d, p->n_in, v->W_emb, v->b_emb, tok + (int64_t)(t - 1) * p->n_in, c->X[0] + t * d);
  for (int l = 0; l < p->n_layers; ++l) {
    const double* X = c->X[l];
    double* xh1 = c->xh1 + (int64_t)l * n * d;
    double* QKV = c->QKV + (int64_t)l * n * 3 * d;
    double* P = c->P + (int64_t)l * H * n * n;
    double* O = c->O + (int64_t)l * n * d;
    double* M = c->M + (int64_t)l * n * d;
    double* xh2 = c->xh2 + (int64_t)l * n * d;
    double* Z = c->Z + (int64_t)l * n * f;
    double* G = c->G + (int64_t)l * n * f;
    for (int t = 0; t < n; ++t) {
      ln_fwd(d, X + t * d, v->ln1_g[l], v->ln1_b[l], xh1 + t * d, c->r1 + l * n + t, y);
      mv(3 * d, d, v->Wqkv[l], v->bqkv[l], y, QKV + t * 3 * d);
    }
    for (int hh = 0; hh < H; ++hh)
      for (int t = 0; t < n; ++t) {
        double mx = -INFINITY, z = 0.0;
        for (int u = 0; u < n; ++u) {
          double acc = 0.0;
          for (int j = 0; j < dh; ++j) acc += QKV[t * 3 * d + hh * dh + j] * QKV[u * 3 * d + d + hh * dh + j];
          s[u] = acc / sqrt((double)dh);
          if (s[u] > mx) mx = s[u];
        }
        for (int u = 0; u < n; ++u) {
          s[u] = exp(s[u] - mx);
          z += s[u];
        }
        for (int u = 0; u < n; ++u) P[((int64_t)hh * n + t) * n + u] = s[u] / z;
        for (int j = 0; j < dh; ++j) {
          double acc = 0.0;
          for (int u = 0; u < n; ++u) acc += P[((int64_t)hh * n + t) * n + u] * QKV[u * 3 * d + 2 * d + hh * dh + j];
          O[t * d + hh * dh + j] = acc;
        }
      }
    for (int t = 0; t < n; ++t) {
      mv(d, d, v->Wo[l], v->bo[l], O + t * d, M + t * d);
      for (int j = 0; j < d; ++j) M[t * d + j] += X[t * d + j];
      ln_fwd(d, M + t * d, v->ln2_g[l], v->ln2_b[l], xh2 + t * d, c->r2 + l * n + t, y);
      mv(f, d, v->W1[l], v->b1[l], y, Z + (int64_t)t * f);
      for (int j = 0; j < f; ++j) G[(int64_t)t * f + j] = g_gelu(Z[(int64_t)t * f + j]);
      mv(d, f, v->W2[l], v->b2[l], G + (int64_t)t * f, c->X[l + 1] + t * d);
      for (int j = 0; j < d; ++j) c->X[l + 1][t * d + j] += M[t * d + j];
    }
  }
  ln_fwd(d, c->X[p->n_layers], v->lnf_g, v->lnf_b, c->xhf, &c->rf, c->U);
  mv(p->n_out, d, v->Wh, v->bh, c->U, c->out);
  free(y);
  free(s);
}

/* Backward pass of one sample from dL/d(head output); accumulates into g. */
static void tfm_bwd(const oc_tfm_dims* p, const tfm_view* v, const double* tok, const tfm_cache* c,
                    const double* dout, tfm_gview* g) {
  const int d = p->d, H = p->n_heads, dh = p->d / p->n_heads, f = 4 * p->d, n = c->n;
  const double sc = 1.0 / sqrt((double)dh);
  double* dX = (double*)xmalloc(sizeof(double) * n * d);
  double* dM = (double*)xmalloc(sizeof(double) * n * d);
  double* dO = (double*)xmalloc(sizeof(double) * n * d);
  double* dQKV = (double*)xmalloc(sizeof(double) * n * 3 * d);
  double* dY = (double*)xmalloc(sizeof(double) * d);
  double* dZ = (double*)xmalloc(sizeof(double) * f);
  double* y = (double*)xmalloc(sizeof(double) * d);
  double* dP = (double*)xmalloc(sizeof(double) * n);
  /* head and final LayerNorm (token 0 only) */
  outer_add(p->n_out, d, dout, c->U, g->Wh);
  for (int i = 0; i < p->n_out; ++i) g->bh[i] += dout[i];
  memset(dY, 0, sizeof(double) * d);
  mtv_add(p->n_out, d, v->Wh, dout, dY);
  ln_bwd(d, c->xhf, c->rf, v->lnf_g, dY, g->lnf_g, g->lnf_b, dX);
  for (int l = p->n_layers - 1; l >= 0; --l) {
    const double* xh1 = c->xh1 + (int64_t)l * n * d;
    const double* QKV = c->QKV + (int64_t)l * n * 3 * d;
    const double* P = c->P + (int64_t)l * H * n * n;
    const double* O = c->O + (int64_t)l * n * d;
    const double* xh2 = c->xh2 + (int64_t)l * n * d;
    const double* Z = c->Z + (int64_t)l * n * f;
    const double* G = c->G + (int64_t)l * n * f;
    /* feed-forward sub-block: X' = M + W2 gelu(W1 LN2(M) + b1) + b2 */
    memcpy(dM, dX, sizeof(double) * n * d);
    for (int t = 0; t < n; ++t) {
      const double* dx = dX + t * d;
      outer_add(d, f, dx, G + (int64_t)t * f, g->W2[l]);
      for (int j = 0; j < d; ++j) g->b2[l][j] += dx[j];
      memset(dZ, 0, sizeof(double) * f);
      mtv_add(d, f, v->W2[l], dx, dZ);
      for (int j = 0; j < f; ++j) dZ[j] *= g_gelu_grad(Z[(int64_t)t * f + j]);
      for (int j = 0; j < d; ++j) y[j] = xh2[t * d + j] * v->ln2_g[l][j] + v->ln2_b[l][j];
      outer_add(f, d, dZ, y, g->W1[l]);
      for (int j = 0; j < f; ++j) g->b1[l][j] += dZ[j];
      memset(dY, 0, sizeof(double) * d);
      mtv_add(f, d, v->W1[l], dZ, dY);
      ln_bwd(d, xh2 + t * d, c->r2[l * n + t], v->ln2_g[l], dY, g->ln2_g[l], g->ln2_b[l], dM + t * d);
    }
    /* attention sub-block: M = X + Wo attn(LN1(X)) + bo */
    memcpy(dX, dM, sizeof(double) * n * d);
    memset(dO, 0, sizeof(double) * n * d);
    for (int t = 0; t < n; ++t) {
      outer_add(d, d, dM + t * d, O + t * d, g->Wo[l]);
      for (int j = 0; j < d; ++j) g->bo[l][j] += dM[t * d + j];
      mtv_add(d, d, v->Wo[l], dM + t * d, dO + t * d);
    }
    memset(dQKV, 0, sizeof(double) * n * 3 * d);
    for (int hh = 0; hh < H; ++hh)
      for (int t = 0; t < n; ++t) {
        const double* Pt = P + ((int64_t)hh * n + t) * n;
        double dot = 0.0;
        for (int u = 0; u < n; ++u) {
          double acc = 0.0;
          for (int j = 0; j < dh; ++j) acc += dO[t * d + hh * dh + j] * QKV[u * 3 * d + 2 * d + hh * dh + j];
          dP[u] = acc;
          dot += Pt[u] * acc;
          for (int j = 0; j < dh; ++j) dQKV[u * 3 * d + 2 * d + hh * dh + j] += Pt[u] * dO[t * d + hh * dh + j];
        }
        for (int u = 0; u < n; ++u) {
          const double ds = Pt[u] * (dP[u] - dot) * sc;
          for (int j = 0; j < dh; ++j) {
            dQKV[t * 3 * d + hh * dh + j] += ds * QKV[u * 3 * d + d + hh * dh + j];
            dQKV[u * 3 * d + d + hh * dh + j] += ds * QKV[t * 3 * d + hh * dh + j];
          }
        }
      }
    for (int t = 0; t < n; ++t) {
      for (int j = 0; j < d; ++j) y[j] = xh1[t * d + j] * v->ln1_g[l][j] + v->ln1_b[l][j];
      outer_add(3 * d, d, dQKV + t * 3 * d, y, g->Wqkv[l]);
      for (int j = 0; j < 3 * d; ++j) g->bqkv[l][j] += dQKV[t * 3 * d + j];
      memset(dY, 0, sizeof(double) * d);
      mtv_add(3 * d, d, v->Wqkv[l], dQKV + t * 3 * d, dY);
      ln_bwd(d, xh1 + t * d, c->r1[l * n + t], v->ln1_g[l], dY, g->ln1_g[l], g->ln1_b[l], dX + t * d);
    }
  }
  /* embedding of the entity tokens; the recurrent input is data */
  for (int t = 1; t < n; ++t) {
    outer_add(d, p->n_in, dX + t * d, tok + (int64_t)(t - 1) * p->n_in, g->W_emb);
    for (int j = 0; j < d; ++j) g->b_emb[j] += dX[t * d + j];
  }
  free(dX); free(dM); free(dO); free(dQKV); free(dY); free(dZ); free(y); free(dP);
}

/* Forward of n samples: out [n][n_out], h_out [n][d] (optional) = the
 * residual stream at token 0 after the last block. */
void oc_tfm_forward(const oc_tfm_dims* p, const double* params, int32_t n, int32_t n_slots, const double* tokens,
                    const int32_t* n_ent, const double* h_in, double* out, double* h_out) {
  tfm_view v = tfm_split(p, params);
#pragma omp parallel for schedule(dynamic, 4)
  for (int i = 0; i < n; ++i) {
    tfm_cache c;
    int ne = n_ent[i] < 0 ? 0 : (n_ent[i] > n_slots ? n_slots : n_ent[i]);
    cache_alloc(p, 1 + ne, &c);
    tfm_fwd(p, &v, tokens + (int64_t)i * n_slots * p->n_in, h_in + (int64_t)i * p->d, &c);
    for (int j = 0; j < p->n_out; ++j) out[(int64_t)i * p->n_out + j] = c.out[j];
    if (h_out)
      for (int j = 0; j < p->d; ++j) h_out[(int64_t)i * p->d + j] = c.X[p->n_layers][j];
    cache_free(p, &c);
  }
}

/* Per-sample loss and dL/d(head output).
 * kind 0 (actor, PPO): out = logits over n_out actions.
 * kind 1 (critic): out[0] = V.
 * st receives per-sample [loss, entropy, clipped, log pi_old - log pi]. */
static double head_loss(int kind, int n_out, const double* out, int32_t act, double logp_old, double adv,
                        double clip_eps, double ent_coef, double ret, double* dout, double* st) {
  if (kind == 1) {
    const double e = out[0] - ret;
    dout[0] = 2.0 * e;
    st[0] = e * e;
    st[1] = out[0];
    st[2] = st[3] = 0.0;
    return e * e;
  }
  double mx = -INFINITY, z = 0.0;
  for (int j = 0; j < n_out; ++j) mx = out[j] > mx ? out[j] : mx;
  for (int j = 0; j < n_out; ++j) z += exp(out[j] - mx);
  const double lse = mx + log(z);
  double Hn = 0.0;
  for (int j = 0; j < n_out; ++j) {
    const double lp = out[j] - lse;
    Hn -= exp(lp) * lp;
  }
  const double lpa = out[act] - lse;
  const double r = exp(lpa - logp_old);
  const double rc = r < 1.0 - clip_eps ? 1.0 - clip_eps : (r > 1.0 + clip_eps ? 1.0 + clip_eps : r);
  const double s1 = r * adv, s2 = rc * adv;
  /* min(s1, s2); on a tie the unclipped term carries the gradient */
  const double gl = s1 <= s2 ? -adv * r : 0.0; /* dL / d log pi(a) */
  const double loss = -(s1 <= s2 ? s1 : s2) - ent_coef * Hn;
  for (int j = 0; j < n_out; ++j) {
    const double lp = out[j] - lse, pj = exp(lp);
    /* d log pi(a)/dz_j = [j == a] - pi_j;  dH/dz_j = -pi_j (log pi_j + H) */
    dout[j] = gl * ((j == act ? 1.0 : 0.0) - pj) + ent_coef * pj * (lp + Hn);
  }
  st[0] = loss;
  st[1] = Hn;
  st[2] = fabs(r - 1.0) > clip_eps ? 1.0 : 0.0;
  st[3] = logp_old - lpa;
  return loss;
}

/* Mean loss over n samples and its gradient (grad, optional, overwritten)
 * with respect to the parameters.  stats (optional, 4 doubles): means of the
 * per-sample [loss, entropy (actor) or V (critic), clipped fraction,
 * approximate KL]. */
double oc_tfm_loss_grad(const oc_tfm_dims* p, const double* params, int32_t n, int32_t n_slots, const double* tokens,
                        const int32_t* n_ent, const double* h_in, int32_t kind, const int32_t* actions,
                        const double* logp_old, const double* adv, double clip_eps, double ent_coef,
                        const double* ret, double* grad, double* stats) {
  const int64_t np = oc_tfm_param_count(p);
  enum { BLK = 16 };
  tfm_view v = tfm_split(p, params);
  /* per-sample gradients of blocks of BLK samples, added in sample order */
  double* gpart = grad ? (double*)xmalloc(sizeof(double) * np * BLK) : NULL;
  double* st = (double*)xmalloc(sizeof(double) * 4 * (n > 0 ? n : 1));
  if (grad) memset(grad, 0, sizeof(double) * np);
  for (int i0 = 0; i0 < n; i0 += BLK) {
    const int i1 = i0 + BLK < n ? i0 + BLK : n;
    if (gpart) memset(gpart, 0, sizeof(double) * np * BLK);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = i0; i < i1; ++i) {
      tfm_cache c;
      double dout[64];
      int ne = n_ent[i] < 0 ? 0 : (n_ent[i] > n_slots ? n_slots : n_ent[i]);
      const double* tok = tokens + (int64_t)i * n_slots * p->n_in;
      cache_alloc(p, 1 + ne, &c);
      tfm_fwd(p, &v, tok, h_in + (int64_t)i * p->d, &c);
      head_loss(kind, p->n_out, c.out, actions ? actions[i] : 0, logp_old ? logp_old[i] : 0.0, adv ? adv[i] : 0.0,
                clip_eps, ent_coef, ret ? ret[i] : 0.0, dout, st + 4 * i);
      if (gpart) {
        for (int j = 0; j < p->n_out; ++j) dout[j] /= n;
        tfm_gview g = tfm_gsplit(p, gpart + (int64_t)(i - i0) * np);
        tfm_bwd(p, &v, tok, &c, dout, &g);
      }
      cache_free(p, &c);
    }
    if (grad)
      for (int i = i0; i < i1; ++i)
        for (int64_t j = 0; j < np; ++j) grad[j] += gpart[(int64_t)(i - i0) * np + j];
  }
  free(gpart);
  /* sums in sample order (deterministic) */
  double acc[4] = {0, 0, 0, 0};
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 4; ++k) acc[k] += st[4 * i + k];
  free(st);
  if (stats)
    for (int k = 0; k < 4; ++k) stats[k] = acc[k] / n;
  return acc[0] / n;
}

/* Generalized advantage estimation by its definition as a discounted sum of
 * TD errors: delta_t = r_t + gamma (1 - done_t) V_{t+1} - V_t and
 * A_t = sum_{l >= 0} (gamma lambda)^l delta_{t+l}, the sum ending with the
 * first step t+l that ends an episode (done) or at the last step T-1.
 * reward, done [T][E]; value [T+1][E]; adv, ret [T][E]; ret = A + V. */
void oc_gae(int32_t T, int32_t E, const double* reward, const double* value, const int32_t* done, double gamma,
            double lam, double* adv, double* ret) {
  for (int e = 0; e < E; ++e)
    for (int t = 0; t < T; ++t) {
      double a = 0.0, w = 1.0;
      for (int u = t; u < T; ++u) {
        const int64_t i = (int64_t)u * E + e;
        const double nd = done[i] ? 0.0 : 1.0;
        const double delta = reward[i] + gamma * nd * value[(int64_t)(u + 1) * E + e] - value[i];
        a += w * delta;
        if (done[i]) break;
        w *= gamma * lam;
      }
      adv[(int64_t)t * E + e] = a;
      ret[(int64_t)t * E + e] = a + value[(int64_t)t * E + e];
    }
}

/* Critic tokens of env e from the true state (Sec. III-A: true 3D position,
 * velocity and direction of every entity): agents first, then targets,
 * packed from slot 0; each [x/S, y/S, z/S, vx, vy, cos psi, sin psi, kind]
 * with velocity in m/s and kind 1 for an agent, 0 for a target; agents at
 * depth 0 moving at agent_speed.  tokens [E][n_slots][8] (zero padded),
 * n_ent [E] = A_e + T_e. */
void oc_state_tokens(int32_t E, const int32_t* agent_off, const int32_t* target_off, int32_t n_slots, double S,
                     double agent_speed, const double* ax, const double* ay, const double* apsi, const double* tx,
                     const double* ty, const double* tz, const double* tpsi, const double* tspeed, double* tokens,
                     int32_t* n_ent) {
  for (int e = 0; e < E; ++e) {
    double* tk = tokens + (int64_t)e * n_slots * 8;
    memset(tk, 0, sizeof(double) * n_slots * 8);
    int s = 0;
    for (int a = agent_off[e]; a < agent_off[e + 1]; ++a, ++s) {
      double* q = tk + s * 8;
      q[0] = ax[a] / S; q[1] = ay[a] / S; q[2] = 0.0;
      q[3] = agent_speed * cos(apsi[a]); q[4] = agent_speed * sin(apsi[a]);
      q[5] = cos(apsi[a]); q[6] = sin(apsi[a]); q[7] = 1.0;
    }
    for (int k = target_off[e]; k < target_off[e + 1]; ++k, ++s) {
      double* q = tk + s * 8;
      q[0] = tx[k] / S; q[1] = ty[k] / S; q[2] = tz[k] / S;
      q[3] = tspeed[k] * cos(tpsi[k]); q[4] = tspeed[k] * sin(tpsi[k]);
      q[5] = cos(tpsi[k]); q[6] = sin(tpsi[k]); q[7] = 0.0;
    }
    n_ent[e] = s;
  }
}
