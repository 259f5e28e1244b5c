/*
 * tref_mlp.c -- ORACLE (test infrastructure only): the learned EOS guess, a
 * multilayer perceptron 2 -> 64 -> 64 -> 2 with SiLU activations, in FP64.
 * The paper has no learned component; the network maps normalised
 * (log10 rho, log10 e) to normalised (log10 T, log10 P) and only supplies the
 * starting cell of the table inversion, whose result is then fixed by the
 * table itself (Sec. 4.2, runtime map).
 *
 * Parameter layout (TREF_MLP_NPARAM = 4482 doubles):
 *   W1[64][2], b1[64], W2[64][64], b2[64], W3[2][64], b3[2]
 * Loss: L = (1/n) sum_s sum_o (y_so - target_so)^2.
 * The gradient is plain reverse-mode differentiation of that expression.
 */
#include "tref.h"
#include <math.h>
#include <string.h>

#define H TREF_MLP_H

static double sigmoid(double a) { return 1.0 / (1.0 + exp(-a)); }

typedef struct {
  const double *W1, *b1, *W2, *b2, *W3, *b3;
} layers;

static layers unpack(const double *p) {
  layers L;
  L.W1 = p;
  L.b1 = L.W1 + 2 * H;
  L.W2 = L.b1 + H;
  L.b2 = L.W2 + H * H;
  L.W3 = L.b2 + H;
  L.b3 = L.W3 + 2 * H;
  return L;
}

static void forward_one(const layers *L, const double *x, double *a1, double *h1, double *a2,
                        double *h2, double *y) {
  for (int o = 0; o < H; ++o) {
    a1[o] = L->W1[o * 2 + 0] * x[0] + L->W1[o * 2 + 1] * x[1] + L->b1[o];
    h1[o] = a1[o] * sigmoid(a1[o]);
  }
  for (int o = 0; o < H; ++o) {
    double s = L->b2[o];
    for (int i = 0; i < H; ++i) s += L->W2[o * H + i] * h1[i];
    a2[o] = s;
    h2[o] = s * sigmoid(s);
  }
  for (int o = 0; o < 2; ++o) {
    double s = L->b3[o];
    for (int i = 0; i < H; ++i) s += L->W3[o * H + i] * h2[i];
    y[o] = s;
  }
}

void tref_mlp_forward(const double *params, int64_t n, const double *x, double *y) {
  layers L = unpack(params);
  for (int64_t s = 0; s < n; ++s) {
    double a1[H], h1[H], a2[H], h2[H];
    forward_one(&L, x + 2 * s, a1, h1, a2, h2, y + 2 * s);
  }
}

double tref_mlp_loss_grad(const double *params, int64_t n, const double *x, const double *target,
                          double *grad) {
  layers L = unpack(params);
  memset(grad, 0, sizeof(double) * TREF_MLP_NPARAM);
  double *gW1 = grad, *gb1 = gW1 + 2 * H, *gW2 = gb1 + H, *gb2 = gW2 + H * H;
  double *gW3 = gb2 + H, *gb3 = gW3 + 2 * H;
  double loss = 0.0;
  for (int64_t s = 0; s < n; ++s) {
    double a1[H], h1[H], a2[H], h2[H], y[2];
    const double *xs = x + 2 * s, *ts = target + 2 * s;
    forward_one(&L, xs, a1, h1, a2, h2, y);
    double gy[2];
    for (int o = 0; o < 2; ++o) {
      double r = y[o] - ts[o];
      loss += r * r;
      gy[o] = 2.0 * r / (double)n;
    }
    double gh2[H], ga2[H], gh1[H], ga1[H];
    for (int i = 0; i < H; ++i) gh2[i] = 0.0;
    for (int o = 0; o < 2; ++o) {
      gb3[o] += gy[o];
      for (int i = 0; i < H; ++i) {
        gW3[o * H + i] += gy[o] * h2[i];
        gh2[i] += L.W3[o * H + i] * gy[o];
      }
    }
    for (int i = 0; i < H; ++i) {
      double sg = sigmoid(a2[i]);
      ga2[i] = gh2[i] * sg * (1.0 + a2[i] * (1.0 - sg));
      gh1[i] = 0.0;
    }
    for (int o = 0; o < H; ++o) {
      gb2[o] += ga2[o];
      for (int i = 0; i < H; ++i) {
        gW2[o * H + i] += ga2[o] * h1[i];
        gh1[i] += L.W2[o * H + i] * ga2[o];
      }
    }
    for (int i = 0; i < H; ++i) {
      double sg = sigmoid(a1[i]);
      ga1[i] = gh1[i] * sg * (1.0 + a1[i] * (1.0 - sg));
    }
    for (int o = 0; o < H; ++o) {
      gb1[o] += ga1[o];
      gW1[o * 2 + 0] += ga1[o] * xs[0];
      gW1[o * 2 + 1] += ga1[o] * xs[1];
    }
  }
  return loss / (double)n;
}
