/* QoZ oracle, learned tuner: the 64 features of the sampled blocks and the
 * 64-128-128-16 ReLU network (forward pass, summed per-head softmax
 * cross-entropy, its gradient by backpropagation, Adam).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU baseline, never by the product path.
 *
 * The paper's concluding section names better selection policies and
 * hyper-parameter auto-tuning as future work; it prints no features or
 * network.  What is computed here is this project's
 * definition, written plainly in double precision.  Parity unpinned against
 * the paper, which fixes no number for it: the tests pin these definitions
 * to closed forms (features of linear, quadratic and trilinear fields; a
 * hand-worked forward pass; Adam's first two steps) and to finite
 * differences of the loss.
 *
 * Features, over the sampled blocks of Sec. 6.1 (each block on its own; no
 * difference reaches across a block's faces), with e = rel_eb * vrange
 * (1 if that is 0) and log-scaling L(v) = log2(1 + v / e):
 *   [0]      log10(rel_eb)
 *   [1]      log10(vrange / sigma), sigma the population deviation of the
 *            sampled values (0 when either is 0)
 *   [2]      ndims / 3
 *   [3]      log2(N) / 30, N the field's points
 *   [4..6]   L(mean |x[p + u_k] - x[p]|) along the field's axes k (2-D: the
 *            third slot is 0)
 *   [7..9]   L(mean |x[p + u_k] - 2 x[p] + x[p - u_k]|) along k
 *   [10..33] fractions of the points in 24 bins of floor(log2 g) + 12
 *            (clamped to [0, 23]; g = 0 in bin 0), g = |forward-difference
 *            gradient| / e
 *   [34..57] the same bins for |x - Lorenzo prediction| / e (the 2-D or 3-D
 *            first-order Lorenzo predictor from the backward neighbours)
 *   [58..60] L(mean |x - linear interpolation|) at half-strides h = 1, 2, 4
 *   [61..63] L(mean |x - cubic interpolation|) at h = 1, 2, 4
 * The interpolation residuals use the stencils of the predictor (Sec. 5.1)
 * on targets at block-local coordinate i = h (mod 2h) along each axis with
 * all four neighbours i +- h, i +- 3h inside the block.
 * Arithmetic: every difference, prediction, product and bin argument is a
 * binary32 operation in the order written here (the sums of many terms are
 * double); 1/e and 1/e^2 are rounded to binary32 once.  The gradient bin is
 * floor(floor(log2(t)) / 2) + 12 with t = |gradient|^2 / e^2, which equals
 * floor(log2(|gradient| / e)) + 12 without a square root; floor(log2) comes
 * from frexp, which is exact.
 *
 * Network: z = (f - mean) / std (std 0 taken as 1); h1 = relu(W1 z + b1);
 * h2 = relu(W2 h1 + b2); o = W3 h2 + b3; heads o[0:2] interpolator,
 * o[2:8] dimension order, o[8:13] alpha, o[13:16] beta; the loss of a sample
 * is the sum over heads of -log softmax(head)[label]; a batch's loss is the
 * mean.  Parameters are packed W1 (128 x 64, row-major), b1, W2 (128 x 128),
 * b2, W3 (16 x 128), b3.  Adam as published by Kingma and Ba (bias-corrected
 * moments). */
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "qoz_oracle.h"

namespace {

int clamp_bin(int b) { return b < 0 ? 0 : (b > 23 ? 23 : b); }

// floor(log2 r) + 12 for a residual ratio r (0 -> bin 0)
int res_bin(float r) {
  if (!(r > 0.0f)) return 0;
  if (std::isinf(r)) return 23;
  int ex = 0;
  std::frexp(r, &ex);  // r = m 2^ex, m in [0.5, 1): floor(log2 r) = ex - 1
  return clamp_bin(ex - 1 + 12);
}

// floor(log2 sqrt(t)) + 12 = floor(floor(log2 t) / 2) + 12 for t = g^2
int grad_bin(float t) {
  if (!(t > 0.0f)) return 0;
  if (std::isinf(t)) return 23;
  int ex = 0;
  std::frexp(t, &ex);
  const int k = ex - 1;
  const int half = k >= 0 ? k / 2 : -((-k + 1) / 2);
  return clamp_bin(half + 12);
}

double lscale(double v, double e) { return std::log2(1.0 + v / e); }

const int kHeadOff[4] = {0, 2, 8, 13};
const int kHeadLen[4] = {2, 6, 5, 3};

}  // namespace

extern "C" {

int orc_features(const float* x, int ndims, const int64_t* dims, double rel_eb, double vrange,
                 const int64_t* origins, int64_t nblocks, const int64_t* block_dims,
                 double* out) {
  if (ndims != 2 && ndims != 3) return 1;
  int64_t N = 1;
  for (int k = 0; k < ndims; ++k) N *= dims[k];
  int64_t st[3];
  st[ndims - 1] = 1;
  for (int k = ndims - 2; k >= 0; --k) st[k] = st[k + 1] * dims[k + 1];
  const double e0 = rel_eb * vrange;
  const double e = e0 > 0.0 ? e0 : 1.0;
  for (int i = 0; i < ORC_NFEAT; ++i) out[i] = 0.0;

  // block-local point p -> field index
  auto at = [&](int64_t b, const int64_t* c) {
    int64_t idx = 0;
    for (int k = 0; k < ndims; ++k) idx += (origins[3 * b + k] + c[k]) * st[k];
    return x[idx];
  };
  const float inv_e = (float)(1.0 / e);
  const float inv_e2 = (float)(1.0 / (e * e));
  const int64_t* bd = block_dims;
  int64_t bpts = 1;
  for (int k = 0; k < ndims; ++k) bpts *= bd[k];

  // sampled mean and deviation (two passes)
  double sum = 0.0;
  int64_t cnt = 0;
  int64_t c[3];
  for (int64_t b = 0; b < nblocks; ++b)
    for (int64_t p = 0; p < bpts; ++p) {
      int64_t r = p;
      for (int k = ndims - 1; k >= 0; --k) {
        c[k] = r % bd[k];
        r /= bd[k];
      }
      sum += (double)at(b, c);
      ++cnt;
    }
  const double mean = cnt ? sum / (double)cnt : 0.0;
  double ss = 0.0;
  for (int64_t b = 0; b < nblocks; ++b)
    for (int64_t p = 0; p < bpts; ++p) {
      int64_t r = p;
      for (int k = ndims - 1; k >= 0; --k) {
        c[k] = r % bd[k];
        r /= bd[k];
      }
      const double d = (double)at(b, c) - mean;
      ss += d * d;
    }
  const double sigma = cnt ? std::sqrt(ss / (double)cnt) : 0.0;

  out[0] = std::log10(rel_eb);
  out[1] = (sigma > 0.0 && vrange > 0.0) ? std::log10(vrange / sigma) : 0.0;
  out[2] = ndims / 3.0;
  out[3] = std::log2((double)N) / 30.0;

  double d1[3] = {0, 0, 0}, d2[3] = {0, 0, 0};
  int64_t n1[3] = {0, 0, 0}, n2[3] = {0, 0, 0};
  int64_t gh[24] = {0}, lh[24] = {0};
  int64_t ng = 0, nl = 0;
  const double hs[3] = {1.0, 2.0, 4.0};
  double lin[3] = {0, 0, 0}, cub[3] = {0, 0, 0};
  int64_t nint[3] = {0, 0, 0};

  for (int64_t b = 0; b < nblocks; ++b)
    for (int64_t p = 0; p < bpts; ++p) {
      int64_t r = p;
      for (int k = ndims - 1; k >= 0; --k) {
        c[k] = r % bd[k];
        r /= bd[k];
      }
      const float v = at(b, c);
      // first and second differences along each axis
      for (int k = 0; k < ndims; ++k) {
        if (c[k] + 1 < bd[k]) {
          int64_t q[3] = {c[0], c[1], c[2]};
          q[k] += 1;
          const float xq = at(b, q);
          d1[k] += (double)std::fabs(xq - v);
          ++n1[k];
          if (c[k] >= 1) {
            int64_t m[3] = {c[0], c[1], c[2]};
            m[k] -= 1;
            d2[k] += (double)std::fabs((xq + at(b, m)) - 2.0f * v);
            ++n2[k];
          }
        }
      }
      // forward-difference gradient
      bool fwd = true;
      for (int k = 0; k < ndims; ++k) fwd = fwd && c[k] + 1 < bd[k];
      if (fwd) {
        float s = 0.0f;
        for (int k = 0; k < ndims; ++k) {
          int64_t q[3] = {c[0], c[1], c[2]};
          q[k] += 1;
          const float d = at(b, q) - v;
          s = s + d * d;
        }
        ++gh[grad_bin(s * inv_e2)];
        ++ng;
      }
      // Lorenzo residual
      bool bwd = true;
      for (int k = 0; k < ndims; ++k) bwd = bwd && c[k] >= 1;
      if (bwd) {
        float pred;
        if (ndims == 3) {
          auto nb = [&](int dz, int dy, int dx) {
            const int64_t q[3] = {c[0] - dz, c[1] - dy, c[2] - dx};
            return at(b, q);
          };
          const float a = (nb(1, 0, 0) + nb(0, 1, 0)) + nb(0, 0, 1);
          const float bb = (nb(1, 1, 0) + nb(1, 0, 1)) + nb(0, 1, 1);
          pred = (a - bb) + nb(1, 1, 1);
        } else {
          const int64_t qy[3] = {c[0] - 1, c[1], 0}, qx[3] = {c[0], c[1] - 1, 0},
                        qxy[3] = {c[0] - 1, c[1] - 1, 0};
          pred = (at(b, qy) + at(b, qx)) - at(b, qxy);
        }
        ++lh[res_bin(std::fabs(v - pred) * inv_e)];
        ++nl;
      }
      // interpolation residuals at h = 1, 2, 4 along every axis
      for (int j = 0; j < 3; ++j) {
        const int64_t h = (int64_t)hs[j];
        for (int k = 0; k < ndims; ++k) {
          if (c[k] % (2 * h) != h || c[k] - 3 * h < 0 || c[k] + 3 * h > bd[k] - 1) continue;
          int64_t q[3] = {c[0], c[1], c[2]};
          q[k] = c[k] - 3 * h;
          const float a3 = at(b, q);
          q[k] = c[k] - h;
          const float a1 = at(b, q);
          q[k] = c[k] + h;
          const float b1 = at(b, q);
          q[k] = c[k] + 3 * h;
          const float b3 = at(b, q);
          lin[j] += (double)std::fabs(v - (a1 + b1) * 0.5f);
          cub[j] += (double)std::fabs(v - ((9.0f * (a1 + b1)) - (a3 + b3)) * 0.0625f);
          ++nint[j];
        }
      }
    }
  for (int k = 0; k < ndims; ++k) {
    out[4 + k] = n1[k] ? lscale(d1[k] / (double)n1[k], e) : 0.0;
    out[7 + k] = n2[k] ? lscale(d2[k] / (double)n2[k], e) : 0.0;
  }
  for (int i = 0; i < 24; ++i) {
    out[10 + i] = ng ? (double)gh[i] / (double)ng : 0.0;
    out[34 + i] = nl ? (double)lh[i] / (double)nl : 0.0;
  }
  for (int j = 0; j < 3; ++j) {
    out[58 + j] = nint[j] ? lscale(lin[j] / (double)nint[j], e) : 0.0;
    out[61 + j] = nint[j] ? lscale(cub[j] / (double)nint[j], e) : 0.0;
  }
  return 0;
}

static void mlp_sample(const double* P, const double* mean, const double* sd, const double* f,
                       double* z, double* h1, double* h2, double* o) {
  const double* W1 = P;
  const double* b1 = W1 + ORC_H * ORC_NFEAT;
  const double* W2 = b1 + ORC_H;
  const double* b2 = W2 + ORC_H * ORC_H;
  const double* W3 = b2 + ORC_H;
  const double* b3 = W3 + ORC_NOUT * ORC_H;
  for (int i = 0; i < ORC_NFEAT; ++i) {
    const double s = sd[i] != 0.0 ? sd[i] : 1.0;
    z[i] = (f[i] - mean[i]) / s;
  }
  for (int o1 = 0; o1 < ORC_H; ++o1) {
    double a = b1[o1];
    for (int i = 0; i < ORC_NFEAT; ++i) a += W1[o1 * ORC_NFEAT + i] * z[i];
    h1[o1] = a > 0.0 ? a : 0.0;
  }
  for (int o2 = 0; o2 < ORC_H; ++o2) {
    double a = b2[o2];
    for (int i = 0; i < ORC_H; ++i) a += W2[o2 * ORC_H + i] * h1[i];
    h2[o2] = a > 0.0 ? a : 0.0;
  }
  for (int k = 0; k < ORC_NOUT; ++k) {
    double a = b3[k];
    for (int i = 0; i < ORC_H; ++i) a += W3[k * ORC_H + i] * h2[i];
    o[k] = a;
  }
}

void orc_mlp_forward(const double* params, const double* mean, const double* sd,
                     const double* X, int64_t B, double* logits) {
  double z[ORC_NFEAT], h1[ORC_H], h2[ORC_H];
  for (int64_t s = 0; s < B; ++s)
    mlp_sample(params, mean, sd, X + s * ORC_NFEAT, z, h1, h2, logits + s * ORC_NOUT);
}

double orc_mlp_loss_grad(const double* params, const double* mean, const double* sd,
                         const double* X, const int32_t* labels, int64_t B, double* grad) {
  const double* W2 = params + ORC_H * ORC_NFEAT + ORC_H;
  const double* W3 = W2 + ORC_H * ORC_H + ORC_H;
  double* gW1 = grad;
  double* gb1 = gW1 + ORC_H * ORC_NFEAT;
  double* gW2 = gb1 + ORC_H;
  double* gb2 = gW2 + ORC_H * ORC_H;
  double* gW3 = gb2 + ORC_H;
  double* gb3 = gW3 + ORC_NOUT * ORC_H;
  if (grad) memset(grad, 0, sizeof(double) * ORC_NPARAM);
  double loss = 0.0;
  double z[ORC_NFEAT], h1[ORC_H], h2[ORC_H], o[ORC_NOUT], dout[ORC_NOUT], dh2[ORC_H], dh1[ORC_H];
  for (int64_t s = 0; s < B; ++s) {
    mlp_sample(params, mean, sd, X + s * ORC_NFEAT, z, h1, h2, o);
    for (int hd = 0; hd < 4; ++hd) {
      const int off = kHeadOff[hd], len = kHeadLen[hd];
      const int lab = labels[4 * s + hd];
      double mx = o[off];
      for (int j = 1; j < len; ++j) mx = o[off + j] > mx ? o[off + j] : mx;
      double se = 0.0;
      for (int j = 0; j < len; ++j) se += std::exp(o[off + j] - mx);
      loss += (std::log(se) + mx) - o[off + lab];
      for (int j = 0; j < len; ++j)
        dout[off + j] = (std::exp(o[off + j] - mx) / se - (j == lab ? 1.0 : 0.0)) / (double)B;
    }
    if (!grad) continue;
    for (int k = 0; k < ORC_NOUT; ++k) {
      gb3[k] += dout[k];
      for (int i = 0; i < ORC_H; ++i) gW3[k * ORC_H + i] += dout[k] * h2[i];
    }
    for (int i = 0; i < ORC_H; ++i) {
      double a = 0.0;
      for (int k = 0; k < ORC_NOUT; ++k) a += W3[k * ORC_H + i] * dout[k];
      dh2[i] = h2[i] > 0.0 ? a : 0.0;
    }
    for (int o2 = 0; o2 < ORC_H; ++o2) {
      gb2[o2] += dh2[o2];
      for (int i = 0; i < ORC_H; ++i) gW2[o2 * ORC_H + i] += dh2[o2] * h1[i];
    }
    for (int i = 0; i < ORC_H; ++i) {
      double a = 0.0;
      for (int o2 = 0; o2 < ORC_H; ++o2) a += W2[o2 * ORC_H + i] * dh2[o2];
      dh1[i] = h1[i] > 0.0 ? a : 0.0;
    }
    for (int o1 = 0; o1 < ORC_H; ++o1) {
      gb1[o1] += dh1[o1];
      for (int i = 0; i < ORC_NFEAT; ++i) gW1[o1 * ORC_NFEAT + i] += dh1[o1] * z[i];
    }
  }
  return loss / (double)B;
}

void orc_adam_step(double* params, const double* grad, double* m, double* v, int64_t n,
                   int64_t t, double lr, double beta1, double beta2, double eps) {
  const double c1 = 1.0 - std::pow(beta1, (double)t);
  const double c2 = 1.0 - std::pow(beta2, (double)t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
    const double mh = m[i] / c1, vh = v[i] / c2;
    params[i] -= lr * mh / (std::sqrt(vh) + eps);
  }
}

}  /* extern "C" */
