// fit.cu -- the FitManager: minimisation of the NLL over the free parameters.
//
// Paper: the FitManager takes the final PDF and a DataSet, performs the fit and writes the
// fitted values back into the parameter Variables (Fig. 1); the default minimiser is
// Minuit 2 (Sec. 4).  Minuit 2 is not available here, so the minimiser is quasi-Newton
// BFGS (Nocedal & Wright, Numerical Optimization, Algorithm 6.1) with a backtracking
// line search on the sufficient-decrease (Armijo) condition, followed by Newton steps on a
// finite-difference Hessian of the gradient; parameter errors are the square roots of the
// diagonal of that Hessian's inverse.  Convergence: EDM = g^T H^-1 g / 2 below tolerance.
//
// The gradient is either the library's adjoint (goo_nll_grad) or central finite
// differences of goo_nll (the plain path's numerical gradient).  Everything here is host
// logic over the library's NLL entry points; each NLL evaluation runs on the GPU.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "model.cuh"

namespace goo {

namespace {

constexpr int kFitRestarts = 3;  // returns from the Newton phase to the quasi-Newton phase

struct Objective {
  goo_model* model;
  const goo_dataset* ds;
  int precision;
  int gradient;  // GOO_GRAD_*
  int P;
  std::vector<int> free_idx;
  std::vector<double> theta0, scale, work, gfull;
  int n_nll = 0, n_grad = 0;

  // x: scaled free coordinates, theta = theta0 + x * scale.  Returns false if the NLL is
  // not finite (outside the model's domain) or the call failed.
  void to_theta(const double* x) {
    work = theta0;
    for (size_t a = 0; a < free_idx.size(); ++a) work[free_idx[a]] = theta0[free_idx[a]] + x[a] * scale[free_idx[a]];
  }
  bool value(const double* x, double* f) {
    to_theta(x);
    n_nll++;
    double v = 0.0;
    int rc = goo_nll(model, ds, work.data(), precision, &v);
    *f = v;
    return rc == GOO_OK && std::isfinite(v);
  }
  bool value_grad(const double* x, double* f, double* g) {
    const int n = (int)free_idx.size();
    if (gradient == GOO_GRAD_ADJOINT) {
      to_theta(x);
      n_grad++;
      double v = 0.0;
      int rc = goo_nll_grad(model, ds, work.data(), precision, &v, gfull.data());
      if (rc != GOO_OK || !std::isfinite(v)) return false;
      *f = v;
      for (int a = 0; a < n; ++a) g[a] = gfull[free_idx[a]] * scale[free_idx[a]];
      for (int a = 0; a < n; ++a)
        if (!std::isfinite(g[a])) return false;
      return true;
    }
    if (!value(x, f)) return false;
    std::vector<double> xp(x, x + n);
    // central differences in scaled units, step 1e-4 of the parameter scale
    const double h = 1e-4;
    for (int a = 0; a < n; ++a) {
      double fp, fm;
      xp[a] = x[a] + h;
      bool ok = value(xp.data(), &fp);
      xp[a] = x[a] - h;
      ok = ok && value(xp.data(), &fm);
      xp[a] = x[a];
      if (!ok) return false;
      g[a] = (fp - fm) / (2 * h);
    }
    n_grad++;
    return true;
  }
};

// Solves A x = b (n x n, row-major) by Gaussian elimination with partial pivoting; A, b are
// overwritten.  Returns false if singular.
bool solve(int n, std::vector<double>& A, std::vector<double>& b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (!(std::fabs(A[piv * n + c]) > 0)) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      const double f = A[r * n + c] / A[c * n + c];
      if (f == 0.0) continue;
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    double s = b[c];
    for (int k = c + 1; k < n; ++k) s -= A[c * n + k] * b[k];
    b[c] = s / A[c * n + c];
  }
  return true;
}

// Cholesky test: true when the symmetric matrix A (n x n) is positive definite.
bool positive_definite(int n, const std::vector<double>& A) {
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0)) return false;
    L[j * n + j] = std::sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double v = A[i * n + j];
      for (int k = 0; k < j; ++k) v -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = v / L[j * n + j];
    }
  }
  return true;
}

bool invert(int n, const std::vector<double>& A, std::vector<double>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    std::vector<double> M = A, e(n, 0.0);
    e[c] = 1.0;
    if (!solve(n, M, e)) return false;
    for (int r = 0; r < n; ++r) inv[r * n + c] = e[r];
  }
  return true;
}

// Symmetrised central-difference Hessian of the gradient in scaled coordinates, with step
// 1e-3 or, if `steps` is given, steps[a] along coordinate a.
bool hessian(Objective& obj, const std::vector<double>& x, std::vector<double>& H,
             const std::vector<double>* steps = nullptr) {
  const int n = (int)x.size();
  H.assign((size_t)n * n, 0.0);
  std::vector<double> xp = x, gp(n), gm(n);
  for (int a = 0; a < n; ++a) {
    const double h = steps ? (*steps)[a] : 1e-3;
    double f;
    xp[a] = x[a] + h;
    if (!obj.value_grad(xp.data(), &f, gp.data())) return false;
    xp[a] = x[a] - h;
    if (!obj.value_grad(xp.data(), &f, gm.data())) return false;
    xp[a] = x[a];
    for (int b = 0; b < n; ++b) H[a * n + b] = (gp[b] - gm[b]) / (2 * h);
  }
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b) {
      const double v = 0.5 * (H[a * n + b] + H[b * n + a]);
      H[a * n + b] = H[b * n + a] = v;
    }
  return true;
}

}  // namespace
}  // namespace goo

using namespace goo;

extern "C" int goo_fit(goo_model* model, const goo_dataset* ds, double* theta, const int* free_mask,
                       const double* scale, const goo_fit_options* opt_in, double* errors_out, goo_fit_result* res) {
  if (!model || !ds || !theta || !free_mask || !scale || !res) return set_error(GOO_ERR_ARG, "goo_fit: NULL argument");
  goo_fit_options opt;
  if (opt_in) {
    opt = *opt_in;
  } else {
    opt.precision = GOO_F32;
    opt.gradient = GOO_GRAD_ADJOINT;
    opt.max_iter = 500;
    opt.edm_tol = 1e-6;
    opt.polish = 1;
    opt.refine = 1;
  }
  if (opt.max_iter <= 0) opt.max_iter = 500;
  if (!(opt.edm_tol > 0)) opt.edm_tol = 1e-6;
  const auto t0 = std::chrono::steady_clock::now();
  Objective obj;
  obj.model = model;
  obj.ds = ds;
  obj.precision = opt.precision;
  obj.gradient = opt.gradient;
  obj.P = model->n_params;
  obj.theta0.assign(theta, theta + obj.P);
  obj.scale.assign(scale, scale + obj.P);
  obj.gfull.assign(obj.P, 0.0);
  for (int p = 0; p < obj.P; ++p)
    if (free_mask[p]) {
      if (!(scale[p] > 0)) return set_error(GOO_ERR_ARG, "goo_fit: parameter %d is free but its scale is %g", p, scale[p]);
      // the cached lineshape path returns no gradient for masses and widths
      if (model->kind == 1 && opt.gradient == GOO_GRAD_ADJOINT && dalitz_lineshape_param(model, p) &&
          !dalitz_floating(model))
        return set_error(GOO_ERR_STATE, "goo_fit: parameter %d is a resonance mass or width; free lineshape parameters "
                                        "need goo_model_set_lineshapes(model, GOO_LINESHAPE_FLOATING)", p);
      obj.free_idx.push_back(p);
    }
  const int n = (int)obj.free_idx.size();
  std::memset(res, 0, sizeof *res);
  std::vector<double> x(n, 0.0), g(n), xt(n), gt(n), d(n), s(n), y(n), Hinv((size_t)n * n, 0.0), Hy(n);
  double f = 0.0;
  if (!obj.value_grad(x.data(), &f, g.data()))
    return set_error(GOO_ERR_ARG, "goo_fit: the NLL is not finite at the starting point (%s)", goo_last_error());
  for (int a = 0; a < n; ++a) Hinv[a * n + a] = 1.0;
  int status = 1;  // 0 converged, 1 iteration limit, 2 line search failure
  int it = 0;
  double edm = 0.0, best_edm = HUGE_VAL;
  int stale = 0;
  // Newton phase state: the finite-difference Hessian of the gradient and its inverse
  std::vector<double> H, Hi;
  bool have_h = false, h_indefinite = false;
  auto edm_of = [&](const std::vector<double>& gg) {
    double e = 0.0;
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) e += 0.5 * gg[a] * Hi[a * n + b] * gg[b];
    return e;
  };
  const bool refine = opt.refine && opt.polish && opt.precision == GOO_F32 && opt.gradient == GOO_GRAD_ADJOINT;
  // The quasi-Newton phase, then the Newton phase; when the latter ends short of the
  // tolerance or on an indefinite Hessian, the quasi-Newton phase starts again from the
  // current point with that Hessian's inverse (or, if it is indefinite, the inverse of its
  // diagonal magnitudes), at most kFitRestarts times.  On small samples the likelihood can be
  // far from quadratic where the quasi-Newton phase stops, and its curvature estimate poor.
  for (int restart = 0;; ++restart) {
    for (; it < opt.max_iter && n > 0; ++it) {
      for (int a = 0; a < n; ++a) {
        double v = 0.0;
        for (int b = 0; b < n; ++b) v -= Hinv[a * n + b] * g[b];
        d[a] = v;
      }
      double gd = 0.0;
      for (int a = 0; a < n; ++a) gd += g[a] * d[a];
      if (!(gd < 0)) {  // not a descent direction: restart from steepest descent
        for (int a = 0; a < n * n; ++a) Hinv[a] = 0.0;
        for (int a = 0; a < n; ++a) {
          Hinv[a * n + a] = 1.0;
          d[a] = -g[a];
        }
        gd = 0.0;
        for (int a = 0; a < n; ++a) gd += g[a] * d[a];
      }
      edm = -0.5 * gd;
      if (edm < opt.edm_tol) {
        status = 0;
        break;
      }
      // Near the minimum the change of the NLL over a step is smaller than its rounding
      // noise and the line search stops making progress: hand over to the Newton phase,
      // which uses gradients only.
      if (edm < 0.5 * best_edm) {
        best_edm = edm;
        stale = 0;
      } else if (++stale >= 10 && opt.polish) {
        break;
      }
      // backtracking line search on sufficient decrease.  The NLL carries rounding noise
      // (FP32 per-event arithmetic: ~sqrt(N) 1e-7 |log f|), so the decrease test allows a
      // tolerance proportional to |NLL|; convergence itself is decided by the EDM, which uses
      // the (smooth) gradient.
      const double ftol = (obj.precision == GOO_F32 ? 1e-9 : 1e-12) * std::fabs(f);
      double alpha = 1.0, ft = 0.0;
      bool ok = false;
      for (int ls = 0; ls < 60; ++ls) {
        for (int a = 0; a < n; ++a) xt[a] = x[a] + alpha * d[a];
        bool good = obj.gradient == GOO_GRAD_ADJOINT ? obj.value_grad(xt.data(), &ft, gt.data()) : obj.value(xt.data(), &ft);
        if (good && ft <= f + 1e-4 * alpha * gd + ftol) {
          ok = true;
          break;
        }
        // quadratic interpolation of the step, kept within [0.1, 0.5] of the last one
        double next = 0.5 * alpha;
        if (good) {
          const double denom = 2.0 * (ft - f - alpha * gd);
          if (denom > 0) next = -gd * alpha * alpha / denom;
        }
        alpha = std::fmin(0.5 * alpha, std::fmax(0.1 * alpha, next));
      }
      if (!ok) {
        status = 2;
        break;
      }
      if (obj.gradient != GOO_GRAD_ADJOINT && !obj.value_grad(xt.data(), &ft, gt.data())) {
        status = 2;
        break;
      }
      double sy = 0.0, yy = 0.0, ss = 0.0;
      for (int a = 0; a < n; ++a) {
        s[a] = xt[a] - x[a];
        y[a] = gt[a] - g[a];
        sy += s[a] * y[a];
        yy += y[a] * y[a];
        ss += s[a] * s[a];
      }
      if (it == 0 && sy > 0 && yy > 0) {  // scale the initial inverse Hessian (N&W eq. 6.20)
        const double gam = sy / yy;
        for (int a = 0; a < n * n; ++a) Hinv[a] *= gam;
      }
      if (sy > 1e-12 * std::sqrt(yy * ss)) {  // curvature condition; otherwise skip the update
        // H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T
        const double rho = 1.0 / sy;
        for (int a = 0; a < n; ++a) {
          double v = 0.0;
          for (int b = 0; b < n; ++b) v += Hinv[a * n + b] * y[b];
          Hy[a] = v;
        }
        double yHy = 0.0;
        for (int a = 0; a < n; ++a) yHy += y[a] * Hy[a];
        for (int a = 0; a < n; ++a)
          for (int b = 0; b < n; ++b)
            Hinv[a * n + b] += -rho * (Hy[a] * s[b] + s[a] * Hy[b]) + (rho * rho * yHy + rho) * s[a] * s[b];
      }
      if (log_level() >= 2)
        std::fprintf(stderr, "[goo] fit it=%d f=%.10f edm=%.3e alpha=%.3e sy=%.3e\n", it, ft, edm, alpha, sy);
      x = xt;
      g = gt;
      f = ft;
    }
    if (log_level() >= 2) std::fprintf(stderr, "[goo] fit bfgs done it=%d status=%d edm=%.3e\n", it, status, edm);
    // Newton phase and errors from the finite-difference Hessian of the gradient.  A Newton
    // step is accepted when it lowers the EDM computed from the gradient at the new point (the
    // gradient is smooth where the NLL value carries rounding noise); a rejected step is
    // halved up to three times.
    if (n > 0 && refine) {
      // FP64 refinement of an FP32 fit: near the minimum the FP32 gradient's rounding is no
      // longer small against the curvature of a large sample.
      // Newton steps with a fixed inverse Hessian on FP64 gradients, each accepted when the
      // EDM drops; returns false if the FP64 gradient could not be evaluated at x
      std::vector<double> dx(n);
      auto newton = [&]() {
        obj.precision = GOO_F64;
        if (!obj.value_grad(x.data(), &f, g.data())) return false;
        edm = edm_of(g);
        for (int step = 0; step < 6 && edm >= 1e-4 * opt.edm_tol; ++step) {
          for (int a = 0; a < n; ++a) {
            dx[a] = 0.0;
            for (int b = 0; b < n; ++b) dx[a] -= Hi[a * n + b] * g[b];
          }
          bool moved = false;
          for (double t = 1.0; t >= 0.125; t *= 0.5) {
            for (int a = 0; a < n; ++a) xt[a] = x[a] + t * dx[a];
            double ft;
            if (!obj.value_grad(xt.data(), &ft, gt.data())) continue;
            const double e = edm_of(gt);
            if (e < edm) {
              x = xt;
              g = gt;
              f = ft;
              edm = e;
              moved = true;
              break;
            }
          }
          if (log_level() >= 2) std::fprintf(stderr, "[goo] fit refine step=%d edm=%.3e moved=%d\n", step, edm, (int)moved);
          if (!moved) break;
        }
        return true;
      };
      // the Hessian from FP32 gradients when it is positive definite, else (or when the steps
      // stall above the tolerance) from FP64 gradients.  The FP32 differences step a quarter of
      // each parameter's error as BFGS estimates it (at least 1e-3): on a large sample the error
      // is small, and a fixed step would leave the gradient change within the FP32 rounding.
      std::vector<double> hsteps(n);
      for (int a = 0; a < n; ++a) hsteps[a] = std::fmax(1e-3, 0.25 * std::sqrt(std::fmax(Hinv[a * n + a], 0.0)));
      obj.precision = opt.precision;
      bool pd = hessian(obj, x, H, &hsteps) && positive_definite(n, H) && invert(n, H, Hi);
      bool h64 = false;
      if (!pd) {
        obj.precision = GOO_F64;
        pd = hessian(obj, x, H) && positive_definite(n, H) && invert(n, H, Hi);
        h64 = true;
      }
      if (pd && newton()) {
        have_h = true;
        if (edm >= opt.edm_tol && !h64) {
          obj.precision = GOO_F64;
          if (hessian(obj, x, H) && positive_definite(n, H) && invert(n, H, Hi)) {
            h64 = true;
            newton();
          }
        }
        // errors (and the final EDM) from the Hessian at the minimum: FP32 gradients when that
        // Hessian is positive definite (with the fixed step, else the error-scaled steps), else
        // FP64 ones
        std::vector<double> H2, Hi2;
        obj.precision = opt.precision;
        bool pd2 = hessian(obj, x, H2) && positive_definite(n, H2);
        if (!pd2) pd2 = hessian(obj, x, H2, &hsteps) && positive_definite(n, H2);
        obj.precision = GOO_F64;
        if (!pd2) pd2 = hessian(obj, x, H2) && positive_definite(n, H2);
        if (pd2 && invert(n, H2, Hi2)) {
          Hi = Hi2;
          edm = edm_of(g);
        }
      }
      obj.precision = opt.precision;
      break;  // no restarts in the refinement
    }
    if (!(n > 0 && (opt.polish || errors_out))) break;
    {
      bool indefinite = false;
      for (int pass = 0; pass < (opt.polish ? 6 : 1); ++pass) {
        if (!hessian(obj, x, H)) break;
        have_h = invert(n, H, Hi);
        if (!have_h) break;
        edm = edm_of(g);
        if (!opt.polish || (edm >= 0 && edm < 1e-4 * opt.edm_tol)) break;
        if (!positive_definite(n, H)) {  // a Newton step could head for a saddle: restart instead
          indefinite = true;
          break;
        }
        std::vector<double> dx(n, 0.0);
        for (int a = 0; a < n; ++a)
          for (int b = 0; b < n; ++b) dx[a] -= Hi[a * n + b] * g[b];
        bool moved = false;
        for (double t = 1.0; t >= 0.125; t *= 0.5) {
          for (int a = 0; a < n; ++a) xt[a] = x[a] + t * dx[a];
          double ft;
          if (!obj.value_grad(xt.data(), &ft, gt.data())) continue;
          if (edm_of(gt) < edm) {
            x = xt;
            g = gt;
            f = ft;
            moved = true;
            break;
          }
        }
        if (log_level() >= 2) std::fprintf(stderr, "[goo] fit newton pass=%d edm=%.3e moved=%d\n", pass, edm, (int)moved);
        if (!moved) break;
      }
      if (have_h && opt.polish && !indefinite && hessian(obj, x, H) && invert(n, H, Hi)) edm = edm_of(g);  // at the final point
      const bool pd = H.size() == (size_t)n * n && positive_definite(n, H);
      if (opt.polish) h_indefinite = have_h && !pd;
      if (!opt.polish || restart >= kFitRestarts || H.size() != (size_t)n * n || (pd && edm >= 0 && edm < opt.edm_tol))
        break;
      if (log_level() >= 2) std::fprintf(stderr, "[goo] fit restart=%d edm=%.3e pd=%d\n", restart + 1, edm, (int)pd);
      if (pd && have_h) {
        Hinv = Hi;
      } else {
        for (int a = 0; a < n * n; ++a) Hinv[a] = 0.0;
        for (int a = 0; a < n; ++a) Hinv[a * n + a] = 1.0 / std::fmax(std::fabs(H[a * n + a]), 1e-12);
      }
      best_edm = HUGE_VAL;
      stale = 0;
      status = 1;
      if (it >= opt.max_iter) break;  // no quasi-Newton iterations left
    }
  }
  if (n > 0 && have_h && (edm < 0 || h_indefinite)) status = 3;  // the final Hessian is not positive definite
  else if (n > 0 && edm < opt.edm_tol) status = 0;
  else if (status == 0) status = 1;
  obj.to_theta(x.data());
  for (int p = 0; p < obj.P; ++p) theta[p] = obj.work[p];
  if (errors_out) {
    for (int p = 0; p < obj.P; ++p) errors_out[p] = 0.0;
    if (have_h)
      for (int a = 0; a < n; ++a) {
        const double v = Hi[a * n + a];
        errors_out[obj.free_idx[a]] = v > 0 ? std::sqrt(v) * obj.scale[obj.free_idx[a]] : NAN;
      }
  }
  res->nll = f;
  res->edm = edm;
  res->iterations = it;
  res->nll_evals = obj.n_nll;
  res->grad_evals = obj.n_grad;
  res->status = status;
  res->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return GOO_OK;
}
