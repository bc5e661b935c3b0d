/*
 * mlp_oracle.c -- plain FP64 CPU restatement of the transport-data surrogate:
 * a fully connected network 2 -> 128 -> 128 -> 6 with tanh hidden units and
 * a linear output, its mean-squared-error gradient by backpropagation, and
 * the Adam update (Kingma & Ba, "Adam: a method for stochastic
 * optimization", ICLR 2015, Algorithm 1).  The network maps (log10 E/N, O2
 * fraction) to the logarithms of the flux transport data a local-field fluid
 * model reads (Sec. 2.2.4 of the paper: mobility, diffusion, alpha, eta and
 * mean energy versus the field).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the CUDA surrogate
 * kernels are checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product path never does.
 * It shares no code, header or constant with the CUDA library.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -o liboracle_mlp.so mlp_oracle.c -lm
 *
 * Parameter vector theta (one array, this order):
 *   W1[128][2], b1[128], W2[128][128], b2[128], W3[6][128], b3[6]
 * (W[o][i] multiplies input i of unit o), 17670 numbers.
 *
 * Pins (tests/test_oracle_mlp.py): the gradient against central finite
 * differences of the loss; a saturated network whose hidden units are exact
 * signs, so the output is an integer matrix-vector product known exactly;
 * zero hidden weights give the output biases; the first Adam step moves every
 * parameter by lr * g / (|g| + eps); the hidden-unit sign symmetry.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NI 2
#define NH 128
#define NO 6

enum {
    OFF_W1 = 0,
    OFF_B1 = OFF_W1 + NH * NI,
    OFF_W2 = OFF_B1 + NH,
    OFF_B2 = OFF_W2 + NH * NH,
    OFF_W3 = OFF_B2 + NH,
    OFF_B3 = OFF_W3 + NO * NH,
    N_PARAMS = OFF_B3 + NO
};

int orc_mlp_n_params(void) { return N_PARAMS; }

/* One point: hidden activations h1, h2 and output y. */
static void forward_point(const double* th, const double* x, double* h1, double* h2, double* y) {
    const double* W1 = th + OFF_W1;
    const double* b1 = th + OFF_B1;
    const double* W2 = th + OFF_W2;
    const double* b2 = th + OFF_B2;
    const double* W3 = th + OFF_W3;
    const double* b3 = th + OFF_B3;
    for (int o = 0; o < NH; ++o) {
        double z = b1[o];
        for (int i = 0; i < NI; ++i) z += W1[o * NI + i] * x[i];
        h1[o] = tanh(z);
    }
    for (int o = 0; o < NH; ++o) {
        double z = b2[o];
        for (int i = 0; i < NH; ++i) z += W2[o * NH + i] * h1[i];
        h2[o] = tanh(z);
    }
    for (int o = 0; o < NO; ++o) {
        double z = b3[o];
        for (int i = 0; i < NH; ++i) z += W3[o * NH + i] * h2[i];
        y[o] = z;
    }
}

/* y[n][6] for x[n][2]. */
void orc_mlp_forward(const double* th, const double* x, int n, double* y) {
    double h1[NH], h2[NH];
    for (int p = 0; p < n; ++p) forward_point(th, x + (size_t)p * NI, h1, h2, y + (size_t)p * NO);
}

/* Loss L = (1 / (6 n)) sum_p sum_o (y_po - t_po)^2 and its gradient with
 * respect to theta, by the chain rule through the layers in reverse:
 *   dy = 2 (y - t) / (6 n);  dW3 += dy h2^T;  db3 += dy
 *   dz2 = (W3^T dy) * (1 - h2^2);  dW2 += dz2 h1^T;  db2 += dz2
 *   dz1 = (W2^T dz2) * (1 - h1^2);  dW1 += dz1 x^T;  db1 += dz1 */
double orc_mlp_loss_grad(const double* th, const double* x, const double* t, int n, double* g) {
    const double* W2 = th + OFF_W2;
    const double* W3 = th + OFF_W3;
    memset(g, 0, sizeof(double) * N_PARAMS);
    double loss = 0.0;
    const double scale = 1.0 / (6.0 * (double)n);
    double h1[NH], h2[NH], y[NO], dy[NO], dz2[NH], dz1[NH];
    for (int p = 0; p < n; ++p) {
        const double* xp = x + (size_t)p * NI;
        const double* tp = t + (size_t)p * NO;
        forward_point(th, xp, h1, h2, y);
        for (int o = 0; o < NO; ++o) {
            const double d = y[o] - tp[o];
            loss += d * d;
            dy[o] = 2.0 * d * scale;
        }
        for (int o = 0; o < NO; ++o) {
            for (int i = 0; i < NH; ++i) g[OFF_W3 + o * NH + i] += dy[o] * h2[i];
            g[OFF_B3 + o] += dy[o];
        }
        for (int i = 0; i < NH; ++i) {
            double s = 0.0;
            for (int o = 0; o < NO; ++o) s += W3[o * NH + i] * dy[o];
            dz2[i] = s * (1.0 - h2[i] * h2[i]);
        }
        for (int o = 0; o < NH; ++o) {
            for (int i = 0; i < NH; ++i) g[OFF_W2 + o * NH + i] += dz2[o] * h1[i];
            g[OFF_B2 + o] += dz2[o];
        }
        for (int i = 0; i < NH; ++i) {
            double s = 0.0;
            for (int o = 0; o < NH; ++o) s += W2[o * NH + i] * dz2[o];
            dz1[i] = s * (1.0 - h1[i] * h1[i]);
        }
        for (int o = 0; o < NH; ++o) {
            for (int i = 0; i < NI; ++i) g[OFF_W1 + o * NI + i] += dz1[o] * xp[i];
            g[OFF_B1 + o] += dz1[o];
        }
    }
    return loss * scale;
}

/* Adam, Algorithm 1 of Kingma & Ba: with step t >= 1,
 *   m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2
 *   m_hat = m / (1 - b1^t);  v_hat = v / (1 - b2^t)
 *   theta <- theta - lr m_hat / (sqrt(v_hat) + eps) */
void orc_mlp_adam(double* th, double* m, double* v, const double* g, int step, double lr, double beta1,
                  double beta2, double eps) {
    const double c1 = 1.0 - pow(beta1, (double)step);
    const double c2 = 1.0 - pow(beta2, (double)step);
    for (int k = 0; k < N_PARAMS; ++k) {
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k];
        v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k];
        const double mh = m[k] / c1, vh = v[k] / c2;
        th[k] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* Full-batch training: n_steps of (gradient, Adam) from the given state;
 * returns the loss before the last update. */
double orc_mlp_train(double* th, double* m, double* v, int step0, const double* x, const double* t, int n,
                     int n_steps, double lr, double beta1, double beta2, double eps) {
    double* g = (double*)malloc(sizeof(double) * N_PARAMS);
    double loss = 0.0;
    for (int s = 0; s < n_steps; ++s) {
        loss = orc_mlp_loss_grad(th, x, t, n, g);
        orc_mlp_adam(th, m, v, g, step0 + s + 1, lr, beta1, beta2, eps);
    }
    free(g);
    return loss;
}
