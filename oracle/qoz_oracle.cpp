/*
 * QoZ oracle, predictor / quantizer / rate / metrics part.
 *
 * TEST INFRASTRUCTURE ONLY (see qoz_oracle.h).  Plain loops over the
 * full-resolution array in the order the paper describes; nothing here is
 * blocked, fused or reordered.  Built with -O2 -ffp-contract=off.
 *
 * Parity pins for each function live in tests/test_oracle_*.py.  The border
 * stencils, the quantizer's rounding rule and the unpredictable-point rule are
 * readings where the paper is silent ("parity unpinned" beyond the
 * polynomial-exactness and error-bound invariants that the tests check).
 */
#include "qoz_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <queue>
#include <utility>
#include <vector>

namespace {

/* Lexicographic permutations of the axes (Sec. 5.2.2 lists 012, 021, 102,
 * 120, 201, 210 for 3D). */
const int kPerm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
const int kPerm2[2][2] = {{0, 1}, {1, 0}};

int log2_exact(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return ((int64_t(1) << l) == v) ? l : -1;
}

/* One-dimensional interpolation along an axis (Sec. 5.1, Sec. 5.2.2).
 * R: reconstructed values; p: linear index of the target; st: element stride
 * of the axis; c: coordinate of the target along the axis; n: axis length;
 * h: half-stride of the level.  Neighbours at c-h and c-3h / c+h, c+3h.
 * Lagrange weights on the equispaced nodes that exist:
 *   cubic  (-a3 + 9 a1 + 9 b1 - b3) / 16
 *   quadratic with a3 (-a3 + 6 a1 + 3 b1) / 8, with b3 (3 a1 + 6 b1 - b3) / 8
 *   linear (a1 + b1) / 2
 *   no right neighbour: linear extrapolation 1.5 a1 - 0.5 a3, else a1. */
float predict_1d(const float* R, int64_t p, int64_t st, int64_t c, int64_t n, int64_t h,
                 int interp) {
  const float a1 = R[p - h * st];
  const bool has_b1 = c + h < n;
  const bool has_a3 = c - 3 * h >= 0;
  const bool has_b3 = c + 3 * h < n;
  if (!has_b1) {
    if (has_a3) {
      const float a3 = R[p - 3 * h * st];
      const float t1 = a1 * 1.5f;
      const float t2 = a3 * 0.5f;
      return t1 - t2;
    }
    return a1;
  }
  const float b1 = R[p + h * st];
  if (interp == 1) {
    if (has_a3 && has_b3) {
      const float a3 = R[p - 3 * h * st];
      const float b3 = R[p + 3 * h * st];
      const float s1 = a1 + b1;
      const float s3 = a3 + b3;
      const float t = 9.0f * s1;
      const float u = t - s3;
      return u * 0.0625f;
    }
    if (has_a3) {
      const float a3 = R[p - 3 * h * st];
      const float t1 = 6.0f * a1;
      const float t2 = 3.0f * b1;
      const float s = t1 + t2;
      const float u = s - a3;
      return u * 0.125f;
    }
    if (has_b3) {
      const float b3 = R[p + 3 * h * st];
      const float t1 = 3.0f * a1;
      const float t2 = 6.0f * b1;
      const float s = t1 + t2;
      const float u = s - b3;
      return u * 0.125f;
    }
  }
  const float s = a1 + b1;
  return s * 0.5f;
}

/* Linear-scale quantization of one point (the quantizer SZ uses, Sec. 5.1):
 * bin width 2 e_l, bin index rounded half away from zero, reconstruction
 * pred + 2 e_l q.  A point is unpredictable when its bin index does not fit
 * in the code range, or when the reconstruction misses the bound (rounding,
 * non-finite values).  Returns true if predictable. */
bool quantize(float x, float pred, float el, float two_e, float inv, uint16_t* code,
              float* rec) {
  const float d = x - pred;
  int q = 0;
  if (d != 0.0f) {
    const float t = std::fabs(d) * inv;
    const float m = std::floor(t + 0.5f);
    if (!(m < 32768.0f)) return false;
    q = (int)m;
    if (d < 0.0f) q = -q;
  }
  const float r = pred + (float)q * two_e;
  if (!(std::fabs(x - r) <= el)) return false;
  *code = (uint16_t)(q + ORC_RADIUS);
  *rec = r;
  return true;
}

struct Field {
  int nd;
  int64_t n[3];   /* slowest-first */
  int64_t st[3];  /* element strides */
  int64_t N;
};

Field make_field(int ndims, const int64_t* dims) {
  Field f;
  f.nd = ndims;
  f.N = 1;
  for (int i = 0; i < ndims; ++i) {
    f.n[i] = dims[i];
    f.N *= dims[i];
  }
  int64_t s = 1;
  for (int i = ndims - 1; i >= 0; --i) {
    f.st[i] = s;
    s *= dims[i];
  }
  return f;
}

bool valid_params(int ndims, const int64_t* dims, const orc_params* p) {
  if (ndims != 2 && ndims != 3) return false;
  for (int i = 0; i < ndims; ++i)
    if (dims[i] < 1) return false;
  const int L = log2_exact(p->anchor_stride);
  if (L < 1 || L > ORC_MAX_LEVELS) return false;
  const int nperm = ndims == 3 ? 6 : 2;
  for (int l = 0; l < L; ++l) {
    if (p->interp[l] > 1) return false;
    if (p->order[l] >= nperm) return false;
  }
  if (!(p->alpha >= 1.0) || !(p->beta >= 1.0)) return false;
  return true;
}

bool is_anchor(const Field& f, const int64_t* c, int64_t s) {
  for (int i = 0; i < f.nd; ++i)
    if (c[i] % s != 0) return false;
  return true;
}

/* Visit every target of pass k of level l (Sec. 5.1): along axis ax[k] the
 * coordinate is h mod 2h; along axes interpolated earlier in this level it is
 * 0 mod h; along the later axes it is 0 mod 2h.  Calls fn(linear index,
 * coordinate along the pass axis) in array order. */
template <class Fn>
void for_each_target(const Field& f, const int* ax, int k, int64_t h, Fn fn) {
  int64_t start[3] = {0, 0, 0}, step[3] = {1, 1, 1};
  for (int j = 0; j < f.nd; ++j) {
    const int a = ax[j];
    if (j < k) {
      start[a] = 0;
      step[a] = h;
    } else if (j == k) {
      start[a] = h;
      step[a] = 2 * h;
    } else {
      start[a] = 0;
      step[a] = 2 * h;
    }
  }
  const int a = ax[k];
  if (f.nd == 2) {
    for (int64_t i0 = start[0]; i0 < f.n[0]; i0 += step[0])
      for (int64_t i1 = start[1]; i1 < f.n[1]; i1 += step[1]) {
        const int64_t c[2] = {i0, i1};
        fn(i0 * f.st[0] + i1 * f.st[1], c[a]);
      }
  } else {
    for (int64_t i0 = start[0]; i0 < f.n[0]; i0 += step[0])
      for (int64_t i1 = start[1]; i1 < f.n[1]; i1 += step[1])
        for (int64_t i2 = start[2]; i2 < f.n[2]; i2 += step[2]) {
          const int64_t c[3] = {i0, i1, i2};
          fn(i0 * f.st[0] + i1 * f.st[1] + i2 * f.st[2], c[a]);
        }
  }
}

template <class Fn>
void for_each_point(const Field& f, Fn fn) {
  int64_t c[3] = {0, 0, 0};
  for (int64_t i = 0; i < f.N; ++i) {
    int64_t r = i;
    for (int d = f.nd - 1; d >= 0; --d) {
      c[d] = r % f.n[d];
      r /= f.n[d];
    }
    fn(i, c);
  }
}

}  // namespace

extern "C" {

int64_t orc_value_range(const float* x, int64_t n, float* out_min, float* out_max) {
  int64_t cnt = 0;
  float mn = 0.0f, mx = 0.0f;
  for (int64_t i = 0; i < n; ++i) {
    const float v = x[i];
    if (!std::isfinite(v)) continue;
    if (cnt == 0) {
      mn = v;
      mx = v;
    } else {
      if (v < mn) mn = v;
      if (v > mx) mx = v;
    }
    ++cnt;
  }
  *out_min = mn;
  *out_max = mx;
  return cnt;
}

void orc_level_bounds(double e, double alpha, double beta, int L, double* el) {
  double a = 1.0; /* alpha^(l-1) */
  for (int l = 1; l <= L; ++l) {
    const double den = a < beta ? a : beta;
    el[l - 1] = e / den;
    a = a * alpha;
  }
}

void orc_order_axes(int ndims, int ord, int* axes) {
  for (int i = 0; i < ndims; ++i) axes[i] = ndims == 3 ? kPerm3[ord][i] : kPerm2[ord][i];
}

int64_t orc_anchor_count(int ndims, const int64_t* dims, int anchor_stride) {
  int64_t c = 1;
  for (int i = 0; i < ndims; ++i) c *= (dims[i] + anchor_stride - 1) / anchor_stride;
  return c;
}

int orc_compress(const float* x, int ndims, const int64_t* dims, double e,
                 const orc_params* p, int stop_level,
                 uint16_t* codes, float* recon_out, float* anchors, int64_t* n_anchors,
                 int64_t* unpred_idx, float* unpred_val, int64_t cap, int64_t* n_unpred,
                 orc_level_stats* stats) {
  if (!valid_params(ndims, dims, p) || !(e >= 0.0)) return 1;
  const Field f = make_field(ndims, dims);
  const int64_t s = p->anchor_stride;
  const int L = log2_exact(s);
  if (stop_level < 1) stop_level = 1;

  std::vector<float> R(f.N, 0.0f);
  std::vector<std::pair<int64_t, float>> unp;
  if (stats) std::memset(stats, 0, sizeof(*stats));

  /* Anchor grid: stored losslessly, recon = x (Sec. 5.2.1). */
  int64_t na = 0;
  for_each_point(f, [&](int64_t i, const int64_t* c) {
    if (is_anchor(f, c, s)) {
      R[i] = x[i];
      codes[i] = 0;
      if (anchors) anchors[na] = x[i];
      ++na;
    }
  });
  if (n_anchors) *n_anchors = na;

  double el_d[ORC_MAX_LEVELS];
  orc_level_bounds(e, p->alpha, p->beta, L, el_d);

  /* Levels from the top (largest stride) down to level 1 (Sec. 5.2.2). */
  for (int l = L; l >= stop_level; --l) {
    const int64_t h = int64_t(1) << (l - 1);
    const float el = (float)el_d[l - 1];
    const float two_e = (float)(2.0 * el_d[l - 1]);
    const float inv = (float)(1.0 / (2.0 * el_d[l - 1]));
    int ax[3];
    orc_order_axes(ndims, p->order[l - 1], ax);
    const int interp = p->interp[l - 1];
    for (int k = 0; k < ndims; ++k) {
      const int a = ax[k];
      for_each_target(f, ax, k, h, [&](int64_t i, int64_t c) {
        const float pred = predict_1d(R.data(), i, f.st[a], c, f.n[a], h, interp);
        const float xv = x[i];
        if (stats) {
          /* Algorithm 1 scores the mean |x - pred|; non-finite terms are skipped. */
          const double ad = std::fabs((double)xv - (double)pred);
          if (std::isfinite(ad)) {
            stats->l1[l - 1] += ad;
            stats->cnt[l - 1] += 1;
          }
        }
        uint16_t code;
        float r;
        if (quantize(xv, pred, el, two_e, inv, &code, &r)) {
          codes[i] = code;
          R[i] = r;
        } else {
          codes[i] = 0;
          R[i] = xv;
          unp.push_back({i, xv});
        }
      });
    }
  }

  std::sort(unp.begin(), unp.end(),
            [](const std::pair<int64_t, float>& u, const std::pair<int64_t, float>& v) {
              return u.first < v.first;
            });
  const int64_t nu = (int64_t)unp.size();
  for (int64_t j = 0; j < nu && j < cap; ++j) {
    unpred_idx[j] = unp[j].first;
    unpred_val[j] = unp[j].second;
  }
  *n_unpred = nu;
  if (recon_out) std::memcpy(recon_out, R.data(), sizeof(float) * f.N);
  return 0;
}

int orc_decompress(const uint16_t* codes, int ndims, const int64_t* dims, double e,
                   const orc_params* p, const float* anchors,
                   const int64_t* unpred_idx, const float* unpred_val, int64_t n_unpred,
                   float* out) {
  if (!valid_params(ndims, dims, p) || !(e >= 0.0)) return 1;
  const Field f = make_field(ndims, dims);
  const int64_t s = p->anchor_stride;
  const int L = log2_exact(s);
  for (int64_t j = 1; j < n_unpred; ++j)
    if (!(unpred_idx[j - 1] < unpred_idx[j])) return 2;

  int64_t na = 0;
  for_each_point(f, [&](int64_t i, const int64_t* c) {
    if (is_anchor(f, c, s)) out[i] = anchors[na++];
  });

  double el_d[ORC_MAX_LEVELS];
  orc_level_bounds(e, p->alpha, p->beta, L, el_d);
  int status = 0;
  for (int l = L; l >= 1; --l) {
    const int64_t h = int64_t(1) << (l - 1);
    const float two_e = (float)(2.0 * el_d[l - 1]);
    int ax[3];
    orc_order_axes(ndims, p->order[l - 1], ax);
    const int interp = p->interp[l - 1];
    for (int k = 0; k < ndims; ++k) {
      const int a = ax[k];
      for_each_target(f, ax, k, h, [&](int64_t i, int64_t c) {
        const uint16_t code = codes[i];
        if (code == 0) {
          const int64_t* it = std::lower_bound(unpred_idx, unpred_idx + n_unpred, i);
          if (it == unpred_idx + n_unpred || *it != i) {
            status = 3;
            out[i] = 0.0f;
            return;
          }
          out[i] = unpred_val[it - unpred_idx];
          return;
        }
        const float pred = predict_1d(out, i, f.st[a], c, f.n[a], h, interp);
        const int q = (int)code - ORC_RADIUS;
        out[i] = pred + (float)q * two_e;
      });
    }
  }
  return status;
}

void orc_histogram(const uint16_t* codes, int ndims, const int64_t* dims, int anchor_stride,
                   uint64_t* hist) {
  const Field f = make_field(ndims, dims);
  std::memset(hist, 0, sizeof(uint64_t) * 65536);
  for_each_point(f, [&](int64_t i, const int64_t* c) {
    if (!is_anchor(f, c, anchor_stride)) hist[codes[i]] += 1;
  });
}

uint64_t orc_huffman_bits(const uint64_t* hist, int K) {
  /* Huffman's construction: repeatedly merge the two lightest subtrees.  The
   * total code length sum(count * depth) equals the sum of the weights of all
   * merged (internal) nodes. */
  std::priority_queue<uint64_t, std::vector<uint64_t>, std::greater<uint64_t>> pq;
  for (int i = 0; i < K; ++i)
    if (hist[i] > 0) pq.push(hist[i]);
  if (pq.empty()) return 0;
  if (pq.size() == 1) return pq.top();
  uint64_t bits = 0;
  while (pq.size() > 1) {
    const uint64_t a = pq.top();
    pq.pop();
    const uint64_t b = pq.top();
    pq.pop();
    bits += a + b;
    pq.push(a + b);
  }
  return bits;
}

double orc_autocorr_blocks(const double* e, const int64_t* starts, int64_t nblocks, int64_t k) {
  /* Eq. (ac), two passes: mean and variance of all errors first, then the
   * lag-k products inside each block. */
  const int64_t n = starts[nblocks];
  if (n <= 0) return 0.0;
  double mu = 0.0;
  for (int64_t i = 0; i < n; ++i) mu += e[i];
  mu /= (double)n;
  double var = 0.0;
  for (int64_t i = 0; i < n; ++i) var += (e[i] - mu) * (e[i] - mu);
  var /= (double)n;
  double cov = 0.0;
  int64_t pairs = 0;
  for (int64_t j = 0; j < nblocks; ++j)
    for (int64_t i = starts[j]; i + k < starts[j + 1]; ++i) {
      cov += (e[i] - mu) * (e[i + k] - mu);
      ++pairs;
    }
  if (pairs == 0 || var == 0.0) return 0.0;
  return (cov / (double)pairs) / var;
}

double orc_autocorr(const float* a, const float* b, int64_t n, int64_t k) {
  std::vector<double> e(n > 0 ? n : 0);
  for (int64_t i = 0; i < n; ++i) e[i] = (double)b[i] - (double)a[i];
  const int64_t starts[2] = {0, n > 0 ? n : 0};
  return orc_autocorr_blocks(e.data(), starts, 1, k);
}

double orc_estimate_bits(const uint64_t* hist, int64_t n_unpred, int64_t n_anchors) {
  return (double)orc_huffman_bits(hist, 65536) + 32.0 * (double)n_unpred +
         32.0 * (double)n_anchors;
}

double orc_max_abs_err(const float* a, const float* b, int64_t n) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double d = std::fabs((double)a[i] - (double)b[i]);
    if (d > m || d != d) m = d;  /* NaN propagates */
  }
  return m;
}

double orc_mse(const float* a, const float* b, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double d = (double)a[i] - (double)b[i];
    s += d * d;
  }
  return n > 0 ? s / (double)n : 0.0;
}

double orc_psnr(const float* a, const float* b, int64_t n, double vrange) {
  const double mse = orc_mse(a, b, n);
  if (mse == 0.0) return INFINITY;
  return 20.0 * std::log10(vrange / std::sqrt(mse));
}

double orc_ssim(const float* a, const float* b, int ndims, const int64_t* dims, int win,
                int step, double vrange, int64_t* n_windows, double* sum_out) {
  /* Eq. (ssim), Eq. (ssim2): local means, population variances and the
   * covariance over each window, constants c1 = (k1 L)^2, c2 = (k2 L)^2 with
   * k1 = 0.01, k2 = 0.03 and L the value range. */
  const Field f = make_field(ndims, dims);
  const double c1 = (0.01 * vrange) * (0.01 * vrange);
  const double c2 = (0.03 * vrange) * (0.03 * vrange);
  int64_t cnt[3] = {1, 1, 1};
  for (int d = 0; d < ndims; ++d) cnt[d] = f.n[d] >= win ? (f.n[d] - win) / step + 1 : 0;
  int64_t nw = 1;
  for (int d = 0; d < ndims; ++d) nw *= cnt[d];
  double total = 0.0;
  const int64_t wz = ndims == 3 ? win : 1;
  const double npts = (double)win * (double)win * (ndims == 3 ? (double)win : 1.0);
  for (int64_t w0 = 0; w0 < (ndims == 3 ? cnt[0] : 1); ++w0)
    for (int64_t w1 = 0; w1 < cnt[ndims - 2]; ++w1)
      for (int64_t w2 = 0; w2 < cnt[ndims - 1]; ++w2) {
        double sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0;
        for (int64_t i = 0; i < wz; ++i)
          for (int64_t j = 0; j < win; ++j)
            for (int64_t k = 0; k < win; ++k) {
              int64_t idx;
              if (ndims == 3)
                idx = (w0 * step + i) * f.st[0] + (w1 * step + j) * f.st[1] + (w2 * step + k);
              else
                idx = (w1 * step + j) * f.st[0] + (w2 * step + k);
              const double xv = a[idx], yv = b[idx];
              sx += xv;
              sy += yv;
              sxx += xv * xv;
              syy += yv * yv;
              sxy += xv * yv;
            }
        const double mx = sx / npts, my = sy / npts;
        const double vx = sxx / npts - mx * mx;
        const double vy = syy / npts - my * my;
        const double cxy = sxy / npts - mx * my;
        const double s = ((2.0 * mx * my + c1) * (2.0 * cxy + c2)) /
                         ((mx * mx + my * my + c1) * (vx + vy + c2));
        total += s;
      }
  if (n_windows) *n_windows = nw;
  if (sum_out) *sum_out = total;
  return nw > 0 ? total / (double)nw : NAN;
}

}  /* extern "C" */
