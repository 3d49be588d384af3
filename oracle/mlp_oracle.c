/*
 * mlp_oracle.c -- plain FP64 multilayer perceptron: forward pass, mean-square
 * loss with its gradient by backpropagation, and one Adam step.
 *
 * TEST INFRASTRUCTURE (part of the oracle library): only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark call it.  It shares no
 * code with the CUDA path.
 *
 * Network: dims[0] -> dims[1] -> ... -> dims[L]; hidden layers apply
 * GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2, the last layer is linear.
 * Parameters are packed layer by layer as W_l (dims[l+1] x dims[l], row-major,
 * y = W x + b) followed by b_l (dims[l+1]).
 * Loss: mean over the batch and the outputs of (y - t)^2.
 * Adam (Kingma & Ba 2015): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
 * p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

double orc_gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }

double orc_gelu_grad(double z)
{
    const double pi = 3.14159265358979323846;
    return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * exp(-0.5 * z * z) / sqrt(2.0 * pi);
}

int64_t orc_mlp_param_count(int L, const int* dims)
{
    int64_t n = 0;
    for (int l = 0; l < L; ++l) n += (int64_t)dims[l + 1] * dims[l] + dims[l + 1];
    return n;
}

/* forward for one sample; z[l] (pre-activations) and a[l] (activations,
 * a[0] = x) are written into caller buffers of size sum(dims). */
static void forward_one(int L, const int* dims, const double* params, const double* x, double* a, double* z,
                        int64_t* off)
{
    memcpy(a, x, sizeof(double) * (size_t)dims[0]);
    const double* p = params;
    for (int l = 0; l < L; ++l) {
        const int din = dims[l], dout = dims[l + 1];
        const double* W = p;
        const double* b = p + (int64_t)dout * din;
        const double* ain = a + off[l];
        double* zo = z + off[l + 1];
        double* ao = a + off[l + 1];
        for (int i = 0; i < dout; ++i) {
            double s = b[i];
            for (int j = 0; j < din; ++j) s += W[(int64_t)i * din + j] * ain[j];
            zo[i] = s;
            ao[i] = (l + 1 < L) ? orc_gelu(s) : s;
        }
        p += (int64_t)dout * din + dout;
    }
}

static int64_t* offsets(int L, const int* dims, int64_t* total)
{
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(L + 2));
    off[0] = 0;
    for (int l = 0; l <= L; ++l) off[l + 1] = off[l] + dims[l];
    *total = off[L + 1];
    return off;
}

void orc_mlp_forward(int L, const int* dims, const double* params, int64_t B, const double* X, double* Y)
{
    int64_t tot;
    int64_t* off = offsets(L, dims, &tot);
    double* a = (double*)malloc(sizeof(double) * (size_t)tot);
    double* z = (double*)malloc(sizeof(double) * (size_t)tot);
    for (int64_t s = 0; s < B; ++s) {
        forward_one(L, dims, params, X + s * dims[0], a, z, off);
        memcpy(Y + s * dims[L], a + off[L], sizeof(double) * (size_t)dims[L]);
    }
    free(a);
    free(z);
    free(off);
}

/* Returns the loss; grad (packed like params) receives d loss / d params. */
double orc_mlp_loss_grad(int L, const int* dims, const double* params, int64_t B, const double* X, const double* T,
                         double* grad)
{
    int64_t tot;
    int64_t* off = offsets(L, dims, &tot);
    const int64_t np = orc_mlp_param_count(L, dims);
    double* a = (double*)malloc(sizeof(double) * (size_t)tot);
    double* z = (double*)malloc(sizeof(double) * (size_t)tot);
    double* d = (double*)malloc(sizeof(double) * (size_t)tot); /* dL/dz per layer */
    int64_t* poff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(L + 1));
    poff[0] = 0;
    for (int l = 0; l < L; ++l) poff[l + 1] = poff[l] + (int64_t)dims[l + 1] * dims[l] + dims[l + 1];
    memset(grad, 0, sizeof(double) * (size_t)np);
    const int dL = dims[L];
    const double scale = 1.0 / ((double)B * dL);
    double loss = 0.0;
    for (int64_t s = 0; s < B; ++s) {
        forward_one(L, dims, params, X + s * dims[0], a, z, off);
        const double* t = T + s * dL;
        for (int i = 0; i < dL; ++i) {
            const double e = a[off[L] + i] - t[i];
            loss += e * e * scale;
            d[off[L] + i] = 2.0 * e * scale; /* output layer is linear */
        }
        for (int l = L - 1; l >= 0; --l) {
            const int din = dims[l], dout = dims[l + 1];
            const double* W = params + poff[l];
            double* gW = grad + poff[l];
            double* gb = gW + (int64_t)dout * din;
            const double* dz = d + off[l + 1];
            const double* ain = a + off[l];
            for (int i = 0; i < dout; ++i) {
                gb[i] += dz[i];
                for (int j = 0; j < din; ++j) gW[(int64_t)i * din + j] += dz[i] * ain[j];
            }
            if (l > 0) { /* back through W and the GELU of layer l */
                double* dzin = d + off[l];
                for (int j = 0; j < din; ++j) {
                    double s2 = 0.0;
                    for (int i = 0; i < dout; ++i) s2 += W[(int64_t)i * din + j] * dz[i];
                    dzin[j] = s2 * orc_gelu_grad(z[off[l] + j]);
                }
            }
        }
    }
    free(a);
    free(z);
    free(d);
    free(off);
    free(poff);
    return loss;
}

void orc_adam_step(int64_t n, double* p, const double* g, double* m, double* v, int64_t t, double lr, double b1,
                   double b2, double eps)
{
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
