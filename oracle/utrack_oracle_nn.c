/*
 * FP64 CPU oracle, neural parts: the transformer agent (policy forward) and
 * the learned range-only estimator (MLP forward, backward, Adam).
 *
 * TEST INFRASTRUCTURE ONLY (see utrack_oracle.c).  Shares nothing with the
 * CUDA path.  Weights are inputs (BF16-representable values produced by the
 * seeded input generator); every product and sum here is in double.
 *
 * Transformer agent: Sec. III-B.1 and the Fig. 3 caption (entity vectors
 * embedded as graph vertices, self-attention, an extra recurrent embedding
 * processed jointly, action distribution from an MLP on the transformed
 * recurrent embedding, LayerNorm throughout).  Readings C16: pre-LN blocks,
 * feed-forward width 4d with exact erf-GELU, LayerNorm epsilon 1e-5, a final
 * LayerNorm then a linear head on the recurrent token; the recurrent token's
 * residual stream after the last block is the next step's recurrent state.
 *
 * Estimator: 96 -> 256 -> 256 -> 256 -> 2 MLP with erf-GELU (reading C18),
 * loss = mean over rows and both coordinates of the squared error, Adam with
 * bias correction (Kingma & Ba, ICLR 2015, Algorithm 1).
 *
 * Pins: permutation invariance over entity tokens, a one-token closed form
 * (attention over a single token returns its value row), gradients against
 * central finite differences, Adam against its closed form.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t d, n_layers, n_heads, n_act, n_in;
} oc_policy_dims;

static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }
static double gelu_grad(double x) {
  return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
}

/* y[n] = W[n][k] x[k] + b[n] */
static void linear(int n, int k, const double* W, const double* b, const double* x, double* y) {
  for (int i = 0; i < n; ++i) {
    double acc = b ? b[i] : 0.0;
    for (int j = 0; j < k; ++j) acc += W[(int64_t)i * k + j] * x[j];
    y[i] = acc;
  }
}

static void layer_norm(int d, const double* x, const double* g, const double* b, double* y) {
  double mu = 0.0, var = 0.0;
  for (int i = 0; i < d; ++i) mu += x[i];
  mu /= d;
  for (int i = 0; i < d; ++i) var += (x[i] - mu) * (x[i] - mu);
  var /= d;
  double inv = 1.0 / sqrt(var + 1e-5);
  for (int i = 0; i < d; ++i) y[i] = (x[i] - mu) * inv * g[i] + b[i];
}

/* Number of parameters of the transformer agent, canonical order:
 * W_emb[d][n_in], b_emb[d]; per layer: ln1_g[d], ln1_b[d], Wqkv[3d][d],
 * bqkv[3d], Wo[d][d], bo[d], ln2_g[d], ln2_b[d], W1[4d][d], b1[4d],
 * W2[d][4d], b2[d]; then lnf_g[d], lnf_b[d], Wh[n_act][d], bh[n_act]. */
int64_t oc_policy_param_count(const oc_policy_dims* p) {
  int64_t d = p->d;
  int64_t per_layer = 2 * d + 3 * d * d + 3 * d + d * d + d + 2 * d + 4 * d * d + 4 * d + 4 * d * d + d;
  return d * p->n_in + d + p->n_layers * per_layer + 2 * d + (int64_t)p->n_act * d + p->n_act;
}

/* Forward pass of the transformer agent for n_agents independent agents.
 * tokens [n_agents][n_slots][n_in]; agent i attends over its recurrent
 * token and its first n_ent[i] entity tokens. */
void oc_policy_forward(const oc_policy_dims* p, const double* params, int32_t n_agents, int32_t n_slots,
                       const double* tokens, const int32_t* n_ent, const double* h_in, double* logits,
                       double* h_out) {
  const int d = p->d, H = p->n_heads, dh = p->d / p->n_heads, F4 = 4 * p->d;
#pragma omp parallel for schedule(dynamic, 16)
  for (int ag = 0; ag < n_agents; ++ag) {
    int n = 1 + n_ent[ag];
    double* X = (double*)malloc(sizeof(double) * n * d);
    double* Y = (double*)malloc(sizeof(double) * n * d);
    double* QKV = (double*)malloc(sizeof(double) * n * 3 * d);
    double* O = (double*)malloc(sizeof(double) * n * d);
    double* Z = (double*)malloc(sizeof(double) * F4);
    double* U = (double*)malloc(sizeof(double) * d);
    double* att = (double*)malloc(sizeof(double) * n);
    const double* q = params;
    const double* W_emb = q; q += (int64_t)d * p->n_in;
    const double* b_emb = q; q += d;
    /* token 0: recurrent embedding; tokens 1..n-1: embedded entities */
    for (int j = 0; j < d; ++j) X[j] = h_in[(int64_t)ag * d + j];
    for (int t = 1; t < n; ++t)
      linear(d, p->n_in, W_emb, b_emb, tokens + ((int64_t)ag * n_slots + (t - 1)) * p->n_in, X + t * d);
    for (int l = 0; l < p->n_layers; ++l) {
      const double* ln1_g = q; q += d;
      const double* ln1_b = q; q += d;
      const double* Wqkv = q; q += (int64_t)3 * d * d;
      const double* bqkv = q; q += 3 * d;
      const double* Wo = q; q += (int64_t)d * d;
      const double* bo = q; q += d;
      const double* ln2_g = q; q += d;
      const double* ln2_b = q; q += d;
      const double* W1 = q; q += (int64_t)F4 * d;
      const double* b1 = q; q += F4;
      const double* W2 = q; q += (int64_t)d * F4;
      const double* b2 = q; q += d;
      /* self-attention sub-block */
      for (int t = 0; t < n; ++t) layer_norm(d, X + t * d, ln1_g, ln1_b, Y + t * d);
      for (int t = 0; t < n; ++t) linear(3 * d, d, Wqkv, bqkv, Y + t * d, QKV + t * 3 * d);
      for (int h = 0; h < H; ++h)
        for (int t = 0; t < n; ++t) {
          const double* Qt = QKV + t * 3 * d + h * dh;
          double mx = -INFINITY;
          for (int s = 0; s < n; ++s) {
            const double* Ks = QKV + s * 3 * d + d + h * dh;
            double acc = 0.0;
            for (int j = 0; j < dh; ++j) acc += Qt[j] * Ks[j];
            att[s] = acc / sqrt((double)dh);
            if (att[s] > mx) mx = att[s];
          }
          double Z0 = 0.0;
          for (int s = 0; s < n; ++s) {
            att[s] = exp(att[s] - mx);
            Z0 += att[s];
          }
          for (int j = 0; j < dh; ++j) {
            double acc = 0.0;
            for (int s = 0; s < n; ++s) acc += att[s] / Z0 * QKV[s * 3 * d + 2 * d + h * dh + j];
            O[t * d + h * dh + j] = acc;
          }
        }
      for (int t = 0; t < n; ++t) {
        linear(d, d, Wo, bo, O + t * d, U);
        for (int j = 0; j < d; ++j) X[t * d + j] += U[j];
      }
      /* feed-forward sub-block */
      for (int t = 0; t < n; ++t) {
        layer_norm(d, X + t * d, ln2_g, ln2_b, Y + t * d);
        linear(F4, d, W1, b1, Y + t * d, Z);
        for (int j = 0; j < F4; ++j) Z[j] = gelu(Z[j]);
        linear(d, F4, W2, b2, Z, U);
        for (int j = 0; j < d; ++j) X[t * d + j] += U[j];
      }
    }
    const double* lnf_g = q; q += d;
    const double* lnf_b = q; q += d;
    const double* Wh = q; q += (int64_t)p->n_act * d;
    const double* bh = q;
    if (h_out)
      for (int j = 0; j < d; ++j) h_out[(int64_t)ag * d + j] = X[j];
    layer_norm(d, X, lnf_g, lnf_b, U);
    linear(p->n_act, d, Wh, bh, U, logits + (int64_t)ag * p->n_act);
    free(X); free(Y); free(QKV); free(O); free(Z); free(U); free(att);
  }
}

/* ------------------------------------------------------------------------ */
/* Estimator MLP.  Canonical parameter order: W1[256][96], b1[256],          */
/* W2[256][256], b2[256], W3[256][256], b3[256], W4[2][256], b4[2].          */
/* ------------------------------------------------------------------------ */
#define MLP_IN 96
#define MLP_H 256
#define MLP_OUT 2

int64_t oc_mlp_param_count(void) {
  return (int64_t)MLP_H * MLP_IN + MLP_H + 2 * ((int64_t)MLP_H * MLP_H + MLP_H) + (int64_t)MLP_OUT * MLP_H + MLP_OUT;
}

typedef struct {
  const double *W[4], *b[4];
} mlp_view;

static mlp_view mlp_split(const double* params) {
  mlp_view v;
  const int nin[4] = {MLP_IN, MLP_H, MLP_H, MLP_H}, nout[4] = {MLP_H, MLP_H, MLP_H, MLP_OUT};
  const double* q = params;
  for (int l = 0; l < 4; ++l) {
    v.W[l] = q; q += (int64_t)nout[l] * nin[l];
    v.b[l] = q; q += nout[l];
  }
  return v;
}

/* Forward: out[B][2].  If pre != NULL it receives the three hidden
 * pre-activations [3][B][256] (for the backward pass). */
void oc_mlp_forward(int32_t B, const double* params, const double* X, double* out, double* pre) {
  mlp_view v = mlp_split(params);
#pragma omp parallel for schedule(static)
  for (int r = 0; r < B; ++r) {
    double a[MLP_H], z[MLP_H], in[MLP_H];
    const double* x = X + (int64_t)r * MLP_IN;
    int nin = MLP_IN;
    for (int j = 0; j < MLP_IN; ++j) in[j] = x[j];
    for (int l = 0; l < 3; ++l) {
      linear(MLP_H, nin, v.W[l], v.b[l], in, z);
      if (pre)
        for (int j = 0; j < MLP_H; ++j) pre[((int64_t)l * B + r) * MLP_H + j] = z[j];
      for (int j = 0; j < MLP_H; ++j) a[j] = gelu(z[j]);
      memcpy(in, a, sizeof(a));
      nin = MLP_H;
    }
    linear(MLP_OUT, MLP_H, v.W[3], v.b[3], in, out + (int64_t)r * MLP_OUT);
  }
}

/* Per-output loss rho(e) of the residual e = out - y and its derivative:
 * delta == 0, rho = e^2 / 2 (squared error); delta > 0, the Huber loss
 * (Huber 1964): e^2 / 2 for |e| <= delta, delta (|e| - delta / 2) beyond. */
static double loss_rho(double e, double delta, double* drho) {
  double ae = fabs(e);
  if (delta > 0.0 && ae > delta) {
    *drho = e > 0.0 ? delta : -delta;
    return delta * (ae - 0.5 * delta);
  }
  *drho = e;
  return 0.5 * e * e;
}

/* Loss L = (1/B) sum_r sum_c rho(out_rc - y_rc) (rho of loss_rho; with
 * delta == 0 that is (1/(2B)) sum (out - y)^2) and its gradient with respect
 * to every parameter (same layout as params).  Returns L. */
double oc_mlp_loss_grad(int32_t B, const double* params, const double* X, const double* Y, double* grad,
                        double delta) {
  mlp_view v = mlp_split(params);
  int64_t np = oc_mlp_param_count();
  double* pre = (double*)malloc(sizeof(double) * 3 * (size_t)B * MLP_H);
  double* out = (double*)malloc(sizeof(double) * (size_t)B * MLP_OUT);
  oc_mlp_forward(B, params, X, out, pre);
  memset(grad, 0, sizeof(double) * np);
  double* gW[4];
  double* gb[4];
  {
    const int nin[4] = {MLP_IN, MLP_H, MLP_H, MLP_H}, nout[4] = {MLP_H, MLP_H, MLP_H, MLP_OUT};
    double* q = grad;
    for (int l = 0; l < 4; ++l) {
      gW[l] = q; q += (int64_t)nout[l] * nin[l];
      gb[l] = q; q += nout[l];
    }
  }
  double loss = 0.0;
  for (int r = 0; r < B; ++r) {
    double dout[MLP_OUT], dz[MLP_H], da[MLP_H];
    for (int c = 0; c < MLP_OUT; ++c) {
      double e = out[(int64_t)r * MLP_OUT + c] - Y[(int64_t)r * MLP_OUT + c], drho;
      loss += loss_rho(e, delta, &drho);
      dout[c] = drho / B;
    }
    /* layer 4 (linear head) */
    const double* z3 = pre + ((int64_t)2 * B + r) * MLP_H;
    for (int c = 0; c < MLP_OUT; ++c) {
      gb[3][c] += dout[c];
      for (int j = 0; j < MLP_H; ++j) gW[3][c * MLP_H + j] += dout[c] * gelu(z3[j]);
    }
    for (int j = 0; j < MLP_H; ++j) {
      double acc = 0.0;
      for (int c = 0; c < MLP_OUT; ++c) acc += dout[c] * v.W[3][c * MLP_H + j];
      da[j] = acc;
    }
    /* hidden layers 3, 2, 1 */
    for (int l = 2; l >= 0; --l) {
      const double* z = pre + ((int64_t)l * B + r) * MLP_H;
      for (int j = 0; j < MLP_H; ++j) dz[j] = da[j] * gelu_grad(z[j]);
      int nin = l == 0 ? MLP_IN : MLP_H;
      const double* zin = l == 0 ? NULL : pre + ((int64_t)(l - 1) * B + r) * MLP_H;
      const double* xin = X + (int64_t)r * MLP_IN;
      for (int j = 0; j < MLP_H; ++j) {
        gb[l][j] += dz[j];
        for (int i = 0; i < nin; ++i) {
          double ain = l == 0 ? xin[i] : gelu(zin[i]);
          gW[l][(int64_t)j * nin + i] += dz[j] * ain;
        }
      }
      if (l > 0)
        for (int i = 0; i < nin; ++i) {
          double acc = 0.0;
          for (int j = 0; j < MLP_H; ++j) acc += dz[j] * v.W[l][(int64_t)j * nin + i];
          da[i] = acc;
        }
    }
  }
  free(pre);
  free(out);
  return loss / B;
}

/* One Adam step (Kingma & Ba 2015, Algorithm 1) at iteration t >= 1. */
void oc_adam(int64_t n, double* theta, double* m, double* v, const double* grad, int32_t t, double lr,
             double beta1, double beta2, double eps) {
  double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    theta[i] -= lr * mh / (sqrt(vh) + eps);
  }
}
