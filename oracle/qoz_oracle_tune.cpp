/*
 * QoZ oracle, online tuning part (Sec. 6).
 *
 * TEST INFRASTRUCTURE ONLY (see qoz_oracle.h).  Each sampled block is cut out
 * and run through orc_compress as an independent small field, one block after
 * the other, exactly as Sec. 6.1 describes; the codes of all blocks are pooled
 * into one histogram for the rate estimate.
 *
 * Readings where the paper is silent or ambiguous (parity unpinned beyond the
 * unit cases in tests/test_oracle_tune.py):
 *   - blocks hold b+1 points per axis, stride S = round(b r^(-1/d)); a block
 *     is predicted with log2 min(b, s) levels, its corners being its anchors;
 *   - Algorithm 1 trials use e_l = e on every level and are greedy from the
 *     top level down; a candidate replaces the best only when its mean L1 is
 *     lower by more than 1e-12 relative;
 *   - Table I: case 3 reruns II at 0.8 e, case 4 at 1.2 e (the table's
 *     assignment); I is kept when it lies on or above the line through II's
 *     two points;
 *   - the target mode (finite target PSNR / SSIM) is this project's
 *     extension: each (alpha, beta) is scored by the bit rate interpolated at
 *     the target on the line through two sampled points, and a short secant on
 *     log e then sets the bound.
 */
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "qoz_oracle.h"

namespace {

int ilog2_floor(int64_t v) {
  int l = 0;
  while ((int64_t(2) << l) <= v) ++l;
  return l;
}

/* Candidate interpolators in enumeration order: linear before cubic, then the
 * dimension orders (all, or only increasing/decreasing). */
void candidate_list(int ndims, int n_orders, std::vector<std::pair<int, int>>* out) {
  out->clear();
  std::vector<int> orders;
  if (ndims == 2) {
    orders = {0, 1};
  } else if (n_orders >= 6) {
    orders = {0, 1, 2, 3, 4, 5};
  } else {
    orders = {0, 5}; /* 012 and 210 */
  }
  for (int t = 0; t < 2; ++t)
    for (int o : orders) out->push_back({t, o});
}

struct Blocks {
  std::vector<int64_t> origins;
  int64_t nb = 0;
  int64_t bd[3] = {1, 1, 1};
};

}  // namespace

extern "C" {

int64_t orc_sample_blocks(int ndims, const int64_t* dims, int b, double rate,
                          int64_t* origins, int64_t cap, int64_t* block_dims, int64_t* stride) {
  const double S_real = (double)b * std::pow(rate, -1.0 / (double)ndims);
  int64_t S = (int64_t)std::llround(S_real);
  if (S < 1) S = 1;
  if (stride) *stride = S;
  std::vector<int64_t> starts[3];
  for (int a = 0; a < ndims; ++a) {
    for (int64_t o = 0; o + b <= dims[a] - 1; o += S) starts[a].push_back(o);
    if (starts[a].empty()) {
      /* the field is shorter than a block along this axis: use its full extent */
      starts[a].push_back(0);
      block_dims[a] = dims[a];
    } else {
      block_dims[a] = b + 1;
    }
  }
  int64_t nb = 0;
  if (ndims == 2) {
    for (int64_t o0 : starts[0])
      for (int64_t o1 : starts[1]) {
        if (nb < cap) {
          origins[3 * nb + 0] = o0;
          origins[3 * nb + 1] = o1;
          origins[3 * nb + 2] = 0;
        }
        ++nb;
      }
  } else {
    for (int64_t o0 : starts[0])
      for (int64_t o1 : starts[1])
        for (int64_t o2 : starts[2]) {
          if (nb < cap) {
            origins[3 * nb + 0] = o0;
            origins[3 * nb + 1] = o1;
            origins[3 * nb + 2] = o2;
          }
          ++nb;
        }
  }
  return nb;
}

int orc_block_trial(const float* x, int ndims, const int64_t* dims,
                    const int64_t* origins, int64_t nblocks, const int64_t* block_dims,
                    const orc_params* p, double e, int stop_level, int ssim_win, int ssim_step,
                    double vrange, orc_trial* out) {
  std::memset(out, 0, sizeof(*out));
  int64_t bn = 1;
  for (int a = 0; a < ndims; ++a) bn *= block_dims[a];
  std::vector<float> blk(bn), rec(bn);
  std::vector<uint16_t> codes(bn);
  std::vector<int64_t> uidx(bn);
  std::vector<float> uval(bn);
  std::vector<uint64_t> hist(65536, 0), bh(65536);
  std::vector<double> errs;           /* errors of every block, block after block */
  std::vector<int64_t> starts(1, 0);  /* where each block's errors start */
  for (int64_t k = 0; k < nblocks; ++k) {
    const int64_t* o = origins + 3 * k;
    /* cut the block out of the field */
    if (ndims == 3) {
      for (int64_t i = 0; i < block_dims[0]; ++i)
        for (int64_t j = 0; j < block_dims[1]; ++j)
          for (int64_t l = 0; l < block_dims[2]; ++l)
            blk[(i * block_dims[1] + j) * block_dims[2] + l] =
                x[((o[0] + i) * dims[1] + (o[1] + j)) * dims[2] + (o[2] + l)];
    } else {
      for (int64_t i = 0; i < block_dims[0]; ++i)
        for (int64_t j = 0; j < block_dims[1]; ++j)
          blk[i * block_dims[1] + j] = x[(o[0] + i) * dims[1] + (o[1] + j)];
    }
    int64_t na = 0, nu = 0;
    orc_level_stats st;
    const int rc = orc_compress(blk.data(), ndims, block_dims, e, p, stop_level, codes.data(),
                                rec.data(), nullptr, &na, uidx.data(), uval.data(), bn, &nu, &st);
    if (rc != 0) return rc;
    orc_histogram(codes.data(), ndims, block_dims, p->anchor_stride, bh.data());
    for (int s = 0; s < 65536; ++s) hist[s] += bh[s];
    out->n_unpred += nu;
    out->n_anchors += na;
    out->npts += bn;
    for (int l = 0; l < ORC_MAX_LEVELS; ++l) {
      out->stats.l1[l] += st.l1[l];
      out->stats.cnt[l] += st.cnt[l];
    }
    for (int64_t i = 0; i < bn; ++i) errs.push_back((double)rec[i] - (double)blk[i]);
    starts.push_back((int64_t)errs.size());
    const double me = orc_max_abs_err(blk.data(), rec.data(), bn);
    if (me > out->max_err || me != me) out->max_err = me;
    out->sse += orc_mse(blk.data(), rec.data(), bn) * (double)bn;
    if (ssim_win > 0) {
      int64_t nw = 0;
      double ssum = 0.0;
      orc_ssim(blk.data(), rec.data(), ndims, block_dims, ssim_win, ssim_step, vrange, &nw,
               &ssum);
      out->ssim_sum += ssum;
      out->ssim_n += nw;
    }
  }
  out->bits = orc_estimate_bits(hist.data(), out->n_unpred, out->n_anchors);
  out->B = out->npts > 0 ? out->bits / (double)out->npts : 0.0;
  out->ac = orc_autocorr_blocks(errs.data(), starts.data(), nblocks, 1);
  return 0;
}

double orc_trial_metric(const orc_trial* t, int metric, double vrange) {
  if (metric == ORC_METRIC_PSNR) {
    const double mse = t->npts > 0 ? t->sse / (double)t->npts : 0.0;
    if (mse == 0.0) return INFINITY;
    return 20.0 * std::log10(vrange / std::sqrt(mse));
  }
  if (metric == ORC_METRIC_SSIM) return t->ssim_n > 0 ? t->ssim_sum / (double)t->ssim_n : NAN;
  if (metric == ORC_METRIC_AC) return -t->ac;
  return -t->max_err;
}

int orc_table1(double b1, double m1, double b2, double m2, double b2p, double m2p,
               double* second_scale) {
  /* case 1: I has no higher rate and no lower quality */
  if (b1 <= b2 && m1 >= m2) return 0;
  /* case 2: II has no higher rate and no lower quality */
  if (b1 >= b2 && m1 <= m2) return 1;
  const bool case3 = b1 > b2 && m1 > m2;
  if (std::isnan(b2p)) {
    if (second_scale) *second_scale = case3 ? 0.8 : 1.2;
    return -1;
  }
  /* Is I above the line through (b2, m2) and (b2p, m2p)? */
  double m_line;
  if (b2p == b2) {
    m_line = m2 > m2p ? m2 : m2p;
  } else {
    m_line = m2 + (m2p - m2) * (b1 - b2) / (b2p - b2);
  }
  return m1 >= m_line ? 0 : 1;
}

/* Candidate k of the (alpha, beta) search: alpha ascending in the outer
 * loop, beta in the inner one (the paper lists the candidates but not the
 * order it visits them in; this is the order taken here). */
void orc_ab_candidate(const orc_tune_opts* o, int k, double* alpha, double* beta) {
  *alpha = o->alphas[k / o->n_beta];
  *beta = o->betas[k % o->n_beta];
}

/* Sec. 6.3.2: the setting kept over the candidates taken in order.  The
 * incumbent is solution I and each new candidate solution II; when Table I
 * asks for a second point of II (case 3: 0.8 e, case 4: 1.2 e) it comes from
 * retrial.  In the max-error (max-CR) mode only B counts (Sec. 7.2.2): a
 * candidate replaces the incumbent when its rate is strictly lower. */
int orc_select_fixed(int n, const double* B, const double* M, int maxerr_mode,
                     orc_retrial_fn retrial, void* ctx) {
  if (n <= 0) return -1;
  int best = 0;
  for (int k = 1; k < n; ++k) {
    bool replace;
    if (maxerr_mode) {
      replace = B[k] < B[best];
    } else {
      double scale = 0.0;
      int r = orc_table1(B[best], M[best], B[k], M[k], NAN, NAN, &scale);
      if (r < 0) {
        double b2 = 0.0, m2 = 0.0;
        if (!retrial || retrial(ctx, k, scale, &b2, &m2) != 0) return -1;
        r = orc_table1(B[best], M[best], B[k], M[k], b2, m2, &scale);
      }
      replace = r == 1;
    }
    if (replace) best = k;
  }
  return best;
}

/* Target mode (this project's extension of Sec. 6.3): the second point of a
 * candidate is taken at 1.2 e0 when the first already meets the target (a
 * larger bound lowers the rate), else at 0.8 e0. */
double orc_target_scale(double M, double target) { return M >= target ? 1.2 : 0.8; }

/* Bit rate where the line through (B, M) and (B2, M2) reaches the target;
 * with equal metrics the lower rate if the target is met, else +inf. */
double orc_target_rate(double B, double M, double B2, double M2, double target) {
  if (M2 == M) return M >= target ? (B < B2 ? B : B2) : INFINITY;
  return B + (target - M) * (B2 - B) / (M2 - M);
}

/* One secant step on (log e, M) through the last two points a and b toward
 * M = target, clamped to [e0 / 16, e_user].  Returns 0 (no step) when the
 * two metrics are equal or the step lands on b's bound. */
int orc_secant_step(double ea, double ma, double eb, double mb, double target, double e0,
                    double e_user, double* e_next) {
  if (ma == mb) return 0;
  const double le = std::log(eb) + (target - mb) * (std::log(ea) - std::log(eb)) / (ma - mb);
  double en = std::exp(le);
  if (en > e_user) en = e_user;
  if (en < e0 / 16.0) en = e0 / 16.0;
  if (en == eb) return 0;
  *e_next = en;
  return 1;
}

/* The bound finally used: the largest tried bound (not above e_user) whose
 * metric met the target; when none did, the smallest tried bound. */
int orc_target_pick(int n, const double* e, const double* M, double target, double e_user) {
  int pick = -1;
  for (int k = 0; k < n; ++k)
    if (M[k] >= target && e[k] <= e_user && (pick < 0 || e[k] > e[pick])) pick = k;
  if (pick < 0) {
    pick = 0;
    for (int k = 1; k < n; ++k)
      if (e[k] < e[pick]) pick = k;
  }
  return pick;
}

int orc_tune(const float* x, int ndims, const int64_t* dims, double e_user, double vrange,
             int metric, double target, const orc_tune_opts* o, orc_tune_result* out) {
  std::memset(out, 0, sizeof(*out));
  const int64_t s = o->anchor_stride;
  int L = 0;
  while ((int64_t(1) << L) < s) ++L;
  const int64_t bmin = o->block < s ? o->block : s;
  const int Ls = ilog2_floor(bmin); /* Algorithm 1: L = log2 min(b, s) */

  int64_t bd[3] = {1, 1, 1};
  int64_t S = 0;
  const int64_t nb = orc_sample_blocks(ndims, dims, o->block, o->rate, nullptr, 0, bd, &S);
  std::vector<int64_t> origins(3 * nb);
  orc_sample_blocks(ndims, dims, o->block, o->rate, origins.data(), nb, bd, &S);
  out->n_blocks = (int32_t)nb;
  int64_t npts = nb;
  for (int a = 0; a < ndims; ++a) npts *= bd[a];
  out->n_sampled_points = npts;

  /* block predictor: anchors at the block corners, log2 min(b, s) levels */
  orc_params bp;
  std::memset(&bp, 0, sizeof(bp));
  bp.anchor_stride = (int32_t)(int64_t(1) << Ls);
  bp.alpha = 1.0;
  bp.beta = 1.0;

  const bool target_mode = !std::isnan(target);
  if (target_mode && metric == ORC_METRIC_AC) return 1; /* AC has no target mode (reading) */
  double e0 = e_user;
  if (target_mode && metric == ORC_METRIC_PSNR) {
    e0 = vrange * std::sqrt(3.0) * std::pow(10.0, -target / 20.0);
    if (e0 > e_user) e0 = e_user;
  }

  auto trial = [&](const orc_params& p, double e, int stop, orc_trial* t) {
    out->n_trials += 1;
    const int win = metric == ORC_METRIC_SSIM ? o->ssim_win : 0;
    return orc_block_trial(x, ndims, dims, origins.data(), nb, bd, &p, e, stop, win,
                           o->ssim_step, vrange, t);
  };

  /* ---- Algorithm 1: level-adapted interpolator selection ---- */
  std::vector<std::pair<int, int>> cands;
  candidate_list(ndims, o->n_orders, &cands);
  for (int l = Ls; l >= 1; --l) {
    double best = INFINITY;
    int bi = 0;
    for (size_t c = 0; c < cands.size(); ++c) {
      orc_params p = bp;
      p.interp[l - 1] = (uint8_t)cands[c].first;
      p.order[l - 1] = (uint8_t)cands[c].second;
      orc_trial t;
      if (trial(p, e0, l, &t) != 0) return 1;
      const double cur = t.stats.cnt[l - 1] > 0 ? t.stats.l1[l - 1] / (double)t.stats.cnt[l - 1]
                                                 : 0.0;
      if (c == 0 || cur < best - 1e-12 * best) {
        best = cur;
        bi = (int)c;
      }
    }
    bp.interp[l - 1] = (uint8_t)cands[bi].first;
    bp.order[l - 1] = (uint8_t)cands[bi].second;
    out->alg1_score[l - 1] = best;
  }

  /* full-field parameters: levels above the sampled top level copy it */
  orc_params fp;
  std::memset(&fp, 0, sizeof(fp));
  fp.anchor_stride = (int32_t)s;
  for (int l = 1; l <= L; ++l) {
    const int src = l <= Ls ? l : Ls;
    fp.interp[l - 1] = bp.interp[src - 1];
    fp.order[l - 1] = bp.order[src - 1];
  }

  /* ---- alpha / beta search, Sec. 6.3: every candidate at e0, alpha
   * ascending then beta ---- */
  const int nc = o->n_alpha * o->n_beta;
  std::vector<orc_params> cp(nc);
  std::vector<double> cB(nc), cM(nc);
  double best_B = 0.0, best_M = 0.0, best_e = e0;
  int sel = 0;
  struct TP {
    double e, B, M;
  };
  std::vector<TP> best_pts;
  for (int k = 0; k < nc; ++k) {
    cp[k] = bp;
    orc_ab_candidate(o, k, &cp[k].alpha, &cp[k].beta);
    if (target_mode) continue;
    orc_trial t;
    if (trial(cp[k], e0, 1, &t) != 0) return 1;
    cB[k] = t.B;
    cM[k] = orc_trial_metric(&t, metric, vrange);
  }
  if (!target_mode) {
    /* Table I keep-best; a second point of solution II is one more trial */
    struct Ctx {
      decltype(trial)* run;
      const std::vector<orc_params>* cp;
      double e0;
      int metric;
      double vrange;
    } ctx{&trial, &cp, e0, metric, vrange};
    auto retrial = [](void* c, int k, double scale, double* b, double* m) -> int {
      Ctx* x = static_cast<Ctx*>(c);
      orc_trial t2;
      if ((*x->run)((*x->cp)[k], scale * x->e0, 1, &t2) != 0) return 1;
      *b = t2.B;
      *m = orc_trial_metric(&t2, x->metric, x->vrange);
      return 0;
    };
    sel = orc_select_fixed(nc, cB.data(), cM.data(), metric == ORC_METRIC_MAXERR ? 1 : 0,
                           retrial, &ctx);
    if (sel < 0) return 1;
    best_B = cB[sel];
    best_M = cM[sel];
  } else {
    /* each candidate's bit rate at the target, from two sampled points;
     * the lowest (first on ties) is kept */
    double best_score = INFINITY;
    bool have = false;
    for (int k = 0; k < nc; ++k) {
      orc_trial t;
      if (trial(cp[k], e0, 1, &t) != 0) return 1;
      const double B = t.B, M = orc_trial_metric(&t, metric, vrange);
      const double sc = orc_target_scale(M, target);
      orc_trial t2;
      if (trial(cp[k], sc * e0, 1, &t2) != 0) return 1;
      const double B2 = t2.B, M2 = orc_trial_metric(&t2, metric, vrange);
      const double Bstar = orc_target_rate(B, M, B2, M2, target);
      if (!have || Bstar < best_score) {
        have = true;
        best_score = Bstar;
        sel = k;
        best_pts = {{e0, B, M}, {sc * e0, B2, M2}};
      }
    }
  }
  fp.alpha = cp[sel].alpha;
  fp.beta = cp[sel].beta;

  if (target_mode) {
    /* secant on (log e, M) for the chosen setting, at most 4 more trials */
    for (int it = 0; it < 4; ++it) {
      const TP a = best_pts[best_pts.size() - 2];
      const TP b = best_pts[best_pts.size() - 1];
      double en = 0.0;
      if (!orc_secant_step(a.e, a.M, b.e, b.M, target, e0, e_user, &en)) break;
      orc_trial t;
      if (trial(cp[sel], en, 1, &t) != 0) return 1;
      best_pts.push_back({en, t.B, orc_trial_metric(&t, metric, vrange)});
    }
    std::vector<double> pe(best_pts.size()), pm(best_pts.size());
    for (size_t k = 0; k < best_pts.size(); ++k) {
      pe[k] = best_pts[k].e;
      pm[k] = best_pts[k].M;
    }
    const int pick = orc_target_pick((int)best_pts.size(), pe.data(), pm.data(), target, e_user);
    best_e = best_pts[pick].e;
    if (best_e > e_user) best_e = e_user;
    best_B = best_pts[pick].B;
    best_M = best_pts[pick].M;
  } else {
    best_e = e_user;
  }

  out->params = fp;
  out->e = best_e;
  out->B = best_B;
  out->M = best_M;
  return 0;
}

}  /* extern "C" */
