/*
 * mlp_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * Plain FP64 statement of the troubled-cell indicator network and its
 * training step: a 5 -> 32 -> 32 -> 1 perceptron with ReLU hidden layers and a
 * logistic output, trained with the weighted binary cross-entropy on logits
 * and Adam.  The paper has no learned component; this network and its
 * training follow the gated-WENO extension of the solver (a small MLP on a
 * normalised 5-cell stencil deciding whether linear-weight reconstruction is
 * safe in a cell).
 *
 * Parameter vector (1281 values): W1[32][5], b1[32], W2[32][32], b2[32],
 * w3[32], b3 -- rows are output neurons.
 *
 * Loss of one sample (logit z, label y in {0,1}, positive-class weight wp):
 *   l = wp * y * softplus(-z) + (1 - y) * softplus(z),
 * averaged over the batch; dl/dz = wp * y * (sigmoid(z) - 1) + (1 - y) * sigmoid(z).
 * Adam (Kingma & Ba 2015) with bias correction:
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   theta -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 *
 * Only tests/ may load this (through the oracle package).
 */
#include <math.h>
#include <string.h>

#define H 32
#define NIN 5
#define NPAR (H * NIN + H + H * H + H + H + 1)

enum { OW1 = 0, OB1 = H * NIN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H };

int mlp_nparams(void) { return NPAR; }

static double relu(double x) { return x > 0.0 ? x : 0.0; }

static double softplus(double x) {  /* log(1 + e^x), stable */
    return x > 0.0 ? x + log1p(exp(-x)) : log1p(exp(x));
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* Forward pass of one sample: hidden activations and the logit. */
static double forward1(const double* th, const double* x, double* h1, double* h2) {
    for (int j = 0; j < H; j++) {
        double a = th[OB1 + j];
        for (int i = 0; i < NIN; i++) a += th[OW1 + j * NIN + i] * x[i];
        h1[j] = relu(a);
    }
    for (int j = 0; j < H; j++) {
        double a = th[OB2 + j];
        for (int i = 0; i < H; i++) a += th[OW2 + j * H + i] * h1[i];
        h2[j] = relu(a);
    }
    double z = th[OB3];
    for (int i = 0; i < H; i++) z += th[OW3 + i] * h2[i];
    return z;
}

/* Logits of n samples x[n][5]. */
void mlp_forward(const double* th, const double* x, long n, double* z) {
    double h1[H], h2[H];
    for (long s = 0; s < n; s++) z[s] = forward1(th, x + s * NIN, h1, h2);
}

/* Mean weighted BCE over n samples and its gradient g[NPAR] (overwritten). */
double mlp_loss_grad(const double* th, const double* x, const double* y, long n, double wp, double* g) {
    memset(g, 0, sizeof(double) * NPAR);
    double h1[H], h2[H], d1[H], d2[H], loss = 0.0;
    for (long s = 0; s < n; s++) {
        const double* xs = x + s * NIN;
        double z = forward1(th, xs, h1, h2);
        double ys = y[s];
        loss += wp * ys * softplus(-z) + (1.0 - ys) * softplus(z);
        double sg = sigmoid(z);
        double dz = (wp * ys * (sg - 1.0) + (1.0 - ys) * sg) / (double)n;
        g[OB3] += dz;
        for (int i = 0; i < H; i++) {
            g[OW3 + i] += dz * h2[i];
            d2[i] = h2[i] > 0.0 ? dz * th[OW3 + i] : 0.0;
        }
        for (int j = 0; j < H; j++) {
            g[OB2 + j] += d2[j];
            for (int i = 0; i < H; i++) g[OW2 + j * H + i] += d2[j] * h1[i];
        }
        for (int i = 0; i < H; i++) {
            double a = 0.0;
            for (int j = 0; j < H; j++) a += th[OW2 + j * H + i] * d2[j];
            d1[i] = h1[i] > 0.0 ? a : 0.0;
        }
        for (int j = 0; j < H; j++) {
            g[OB1 + j] += d1[j];
            for (int i = 0; i < NIN; i++) g[OW1 + j * NIN + i] += d1[j] * xs[i];
        }
    }
    return loss / (double)n;
}

/* One Adam update at step t (1-based) of parameters th with gradient g. */
void mlp_adam(double* th, const double* g, double* m, double* v, int t, double lr, double b1, double b2,
              double eps) {
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int k = 0; k < NPAR; k++) {
        m[k] = b1 * m[k] + (1.0 - b1) * g[k];
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
        th[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
    }
}

/* Normalised sensor stencil x_k = (v_k - v_2) / max_j |v_j - v_2|.  A stencil
 * whose variation max_j |v_j - v_2| is at most delta |v_2| (a relative
 * round-off floor) is flat: x = 0 and the return value is 0; otherwise 1. */
int mlp_normalise(const double* v5, double delta, double* x) {
    double m = 0.0;
    for (int k = 0; k < 5; k++) {
        double d = fabs(v5[k] - v5[2]);
        if (d > m) m = d;
    }
    if (!(m > delta * fabs(v5[2]))) {
        for (int k = 0; k < 5; k++) x[k] = 0.0;
        return 0;
    }
    for (int k = 0; k < 5; k++) x[k] = (v5[k] - v5[2]) / m;
    return 1;
}
