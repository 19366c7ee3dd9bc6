// api.cu -- the extern "C" model, normalisation and likelihood entry points.
//
// Paper: the FitManager evaluates the final PDF on an unbinned DataSet (Fig. 1); most of the
// time of a fit is the per-event evaluation (Sec. 1); MPI splits the events among processes
// (Sec. 4).
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstring>

#include "common.cuh"
#include "model.cuh"

using namespace goo;

namespace {

int check_model_dataset(const goo_model* m, const goo_dataset* ds, int precision) {
  if (!m || !ds) return set_error(GOO_ERR_ARG, "NULL model or dataset");
  if (ds->ctx != m->ctx) return set_error(GOO_ERR_ARG, "model and dataset belong to different contexts");
  if (precision != GOO_F64 && precision != GOO_F32) return set_error(GOO_ERR_ARG, "precision=%d", precision);
  if (ds->w64 && m->kind != 0)
    return set_error(GOO_ERR_UNSUPPORTED, "per-event weights are supported by sum-of-product models only");
  if (ds->host_borrowed && (m->kind != 0 || precision != GOO_F32))
    return set_error(GOO_ERR_UNSUPPORTED,
                     "a GOO_BORROW_HOST dataset (float32 columns in host memory) serves FP32 evaluations of "
                     "sum-of-product models only");
  if (ds->ncols < m->n_obs)
    return set_error(GOO_ERR_ARG, "dataset has %d columns, model uses %d observables", ds->ncols, m->n_obs);
  for (int o = 0; o < m->n_obs; ++o)
    if (ds->lo[o] != m->lo[o] || ds->hi[o] != m->hi[o])
      return set_error(GOO_ERR_ARG, "observable %d: dataset limits [%g, %g] differ from the model's [%g, %g]", o,
                       ds->lo[o], ds->hi[o], m->lo[o], m->hi[o]);
  return GOO_OK;
}

int check_theta(const goo_model* m, const double* theta) {
  if (!theta) return set_error(GOO_ERR_ARG, "theta is NULL");
  for (int p = 0; p < m->n_params; ++p)
    if (!std::isfinite(theta[p])) return set_error(GOO_ERR_ARG, "theta[%d] is not finite", p);
  return GOO_OK;
}

int nll_common(goo_model* m, const goo_dataset* ds, const double* theta, int precision, bool grad, double* nll_out,
               double* grad_out) {
  GOO_TRY(check_model_dataset(m, ds, precision));
  GOO_TRY(check_theta(m, theta));
  goo_ctx* ctx = m->ctx;
  GOO_CUDA_TRY(cudaSetDevice(ctx->device));
  const int P = m->n_params;
  double res[2 + kMaxParams];
  if (m->kind == 1) {
    GOO_TRY(dalitz_nll(m, ds, 0, ds->n, theta, precision, grad, res, 0));
  } else if (m->kind == 2) {
    GOO_TRY(td4_nll(m, ds, 0, ds->n, theta, precision, grad, res, 0));
  } else {
    const bool fuse = ds->n > 0 && !ds->w64 && sop_norm_in_event(m, precision, grad);
    GOO_TRY(sop_prepare(m, theta, precision, fuse));
    arm_result_mapped(ctx);
    if (ds->n > 0) GOO_TRY(sop_events(m, ds, 0, ds->n, precision, grad, 0, fuse, ctx->scratch.result_host));
    if (ds->n == 0) {
      res[0] = 0.0;
      res[1] = 0.0;
      for (int p = 0; p < P; ++p) res[2 + p] = 0.0;
      GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    } else {
      GOO_TRY(read_result_mapped(ctx, 2 + P, res));
    }
  }
  if (res[1] <= -2) {
    *nll_out = HUGE_VAL;
    if (grad_out)
      for (int p = 0; p < P; ++p) grad_out[p] = 0.0;
    return set_error(GOO_ERR_RANGE, "%.0f events lie outside the observable limits", -res[1] - 2);
  }
  if (res[1] < 0) {
    *nll_out = HUGE_VAL;
    return set_error(GOO_ERR_TIMEOUT, "a device wait for event data gave up; the result is invalid");
  }
  if (res[1] > 0) {
    *nll_out = HUGE_VAL;
    if (grad_out)
      for (int p = 0; p < P; ++p) grad_out[p] = 0.0;
    return set_error(GOO_ERR_NONPOSITIVE_PDF, "density is <= 0 (or not finite) for %.0f events", res[1]);
  }
  *nll_out = res[0];
  if (grad_out)
    for (int p = 0; p < P; ++p) grad_out[p] = res[2 + p];
  return GOO_OK;
}

}  // namespace

extern "C" {

int goo_model_build(goo_ctx* ctx, const goo_node* nodes, int n_nodes, int n_params, int n_obs, const double* obs_lo,
                    const double* obs_hi, goo_model** out) {
  if (!ctx || !nodes || !out || !obs_lo || !obs_hi) return set_error(GOO_ERR_ARG, "goo_model_build: NULL argument");
  *out = nullptr;
  if (n_nodes < 1 || n_nodes > 256) return set_error(GOO_ERR_ARG, "goo_model_build: n_nodes=%d", n_nodes);
  if (n_params < 0 || n_params > kMaxParams)
    return set_error(GOO_ERR_ARG, "goo_model_build: n_params=%d (max %d)", n_params, kMaxParams);
  if (n_obs < 1 || n_obs > kMaxCols) return set_error(GOO_ERR_ARG, "goo_model_build: n_obs=%d (1..%d)", n_obs, kMaxCols);
  for (int o = 0; o < n_obs; ++o)
    if (!(obs_lo[o] < obs_hi[o])) return set_error(GOO_ERR_ARG, "goo_model_build: observable %d has lo >= hi", o);
  for (int i = 0; i < n_nodes; ++i) {
    const goo_node& n = nodes[i];
    if (n.n_child < 0 || n.n_child > GOO_MAX_CHILD)
      return set_error(GOO_ERR_ARG, "goo_model_build: node %d has %d children", i, n.n_child);
    for (int c = 0; c < n.n_child; ++c)
      if (n.child[c] < 0 || n.child[c] >= i)
        return set_error(GOO_ERR_ARG, "goo_model_build: node %d child %d = %d is not an earlier node (post-order)", i,
                         c, n.child[c]);
  }
  GOO_CUDA_TRY(cudaSetDevice(ctx->device));
  goo_model* m = new goo_model();
  m->ctx = ctx;
  m->n_params = n_params;
  m->n_obs = n_obs;
  for (int o = 0; o < n_obs; ++o) {
    m->lo[o] = obs_lo[o];
    m->hi[o] = obs_hi[o];
  }
  int rc;
  if (nodes[n_nodes - 1].op == GOO_OP_COHERENT || nodes[n_nodes - 1].op == GOO_OP_TD3) {
    rc = build_dalitz_model(ctx, nodes, n_nodes, n_params, n_obs, obs_lo, obs_hi, m);
  } else if (nodes[n_nodes - 1].op == GOO_OP_TD4) {
    rc = build_td4_model(ctx, nodes, n_nodes, n_params, n_obs, m);
  } else {
    rc = build_sop_model(ctx, nodes, n_nodes, n_params, n_obs, obs_lo, obs_hi, m);
    m->norm.kind = GOO_NORM_ANALYTIC;
  }
  if (rc != GOO_OK) {
    goo_model_free(m);
    return rc;
  }
  ctx->live++;
  m->counted = true;
  *out = m;
  return GOO_OK;
}

int goo_model_set_norm(goo_model* m, const goo_norm_spec* spec) {
  if (!m || !spec) return set_error(GOO_ERR_ARG, "goo_model_set_norm: NULL argument");
  if (spec->kind == GOO_NORM_MC && spec->mc && spec->mc->host_borrowed)
    return set_error(GOO_ERR_UNSUPPORTED, "goo_model_set_norm: the MC sample cannot be a GOO_BORROW_HOST dataset");
  GOO_CUDA_TRY(cudaSetDevice(m->ctx->device));
  if (m->kind == 2) return td4_set_norm(m, spec);
  return m->kind == 1 ? dalitz_set_norm(m, spec) : sop_set_norm(m, spec);
}

int goo_model_free(goo_model* m) {
  if (!m) return set_error(GOO_ERR_ARG, "goo_model_free: NULL model");
  cudaSetDevice(m->ctx->device);
  cudaStreamSynchronize(m->ctx->stream);
  if (m->dev) cudaFree(m->dev);
  if (m->stage) cudaFreeHost(m->stage);
  if (m->dalitz) dalitz_free(m);
  if (m->td4) td4_free(m);
  if (m->counted) m->ctx->live--;
  delete m;
  return GOO_OK;
}

int goo_model_components(const goo_model* m) {
  if (!m) return set_error(GOO_ERR_ARG, "goo_model_components: NULL model");
  return m->kind >= 1 ? 1 : m->host.nK;
}

int goo_normalise(goo_model* m, const double* theta, int precision, double* norms_out) {
  if (!m || !norms_out) return set_error(GOO_ERR_ARG, "goo_normalise: NULL argument");
  if (precision != GOO_F64 && precision != GOO_F32) return set_error(GOO_ERR_ARG, "precision=%d", precision);
  GOO_TRY(check_theta(m, theta));
  GOO_CUDA_TRY(cudaSetDevice(m->ctx->device));
  if (m->kind == 1) return dalitz_normalise(m, theta, precision, norms_out);
  if (m->kind == 2) return td4_normalise(m, theta, precision, norms_out);
  GOO_TRY(sop_prepare(m, theta, precision));
  goo_ctx* ctx = m->ctx;
  CompDev comp[kMaxComp];
  GOO_CUDA_TRY(cudaMemcpyAsync(comp, (const char*)m->dev + offsetof(ModelDev, comp), sizeof comp,
                               cudaMemcpyDeviceToHost, ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < m->host.nK; ++k) norms_out[k] = std::exp(comp[k].log_norm);
  return GOO_OK;
}

int goo_nll(goo_model* m, const goo_dataset* ds, const double* theta, int precision, double* nll_out) {
  if (!nll_out) return set_error(GOO_ERR_ARG, "goo_nll: nll_out is NULL");
  return nll_common(m, ds, theta, precision, false, nll_out, nullptr);
}

int goo_nll_grad(goo_model* m, const goo_dataset* ds, const double* theta, int precision, double* nll_out,
                 double* grad_out) {
  if (!nll_out || !grad_out) return set_error(GOO_ERR_ARG, "goo_nll_grad: NULL output");
  return nll_common(m, ds, theta, precision, true, nll_out, grad_out);
}

int goo_eval_logf(goo_model* m, const goo_dataset* ds, const double* theta, int precision, double* logf_dev) {
  GOO_TRY(check_model_dataset(m, ds, precision));
  GOO_TRY(check_theta(m, theta));
  if (!logf_dev && ds->n > 0) return set_error(GOO_ERR_ARG, "goo_eval_logf: logf_dev is NULL");
  if (ds->host_borrowed) return set_error(GOO_ERR_UNSUPPORTED, "goo_eval_logf: GOO_BORROW_HOST dataset");
  GOO_CUDA_TRY(cudaSetDevice(m->ctx->device));
  if (m->kind == 1) {
    GOO_TRY(dalitz_eval_logf(m, ds, theta, precision, logf_dev));
  } else if (m->kind == 2) {
    GOO_TRY(td4_eval_logf(m, ds, theta, precision, logf_dev));
  } else {
    GOO_TRY(sop_prepare(m, theta, precision));
    GOO_TRY(sop_eval_logf(m, ds, precision, logf_dev));
  }
  GOO_CUDA_TRY(cudaStreamSynchronize(m->ctx->stream));
  return GOO_OK;
}

int goo_nll_partial(goo_model* m, const goo_dataset* ds, int64_t begin, int64_t end, const double* theta,
                    int precision, int want_grad, double* out) {
  if (!out) return set_error(GOO_ERR_ARG, "goo_nll_partial: out is NULL");
  GOO_TRY(check_model_dataset(m, ds, precision));
  GOO_TRY(check_theta(m, theta));
  if (begin < 0 || end < begin || end > ds->n)
    return set_error(GOO_ERR_ARG, "goo_nll_partial: range [%lld, %lld) of %lld events", (long long)begin,
                     (long long)end, (long long)ds->n);
  GOO_CUDA_TRY(cudaSetDevice(m->ctx->device));
  goo_ctx* ctx = m->ctx;
  const int P = m->n_params;
  double res[3 + kMaxParams];
  if (m->kind == 2) {
    GOO_TRY(td4_nll(m, ds, begin, end, theta, precision, want_grad != 0, res, 1));
  } else if (m->kind == 1) {
    GOO_TRY(dalitz_nll(m, ds, begin, end, theta, precision, want_grad != 0, res, 1));
  } else {
    const bool fuse = end > begin && !ds->w64 && sop_norm_in_event(m, precision, want_grad != 0);
    GOO_TRY(sop_prepare(m, theta, precision, fuse));
    if (end > begin) {
      arm_result_mapped(ctx);
      GOO_TRY(sop_events(m, ds, begin, end, precision, want_grad != 0, 1, fuse, ctx->scratch.result_host));
      GOO_TRY(read_result_mapped(ctx, 3 + P, res));
    } else {
      GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      for (int i = 0; i < 3 + P; ++i) res[i] = 0.0;
    }
  }
  const double nbad = res[2];
  out[0] = res[0];
  out[1] = res[1];
  out[2] = (double)(end - begin);
  for (int p = 0; p < P; ++p) out[3 + p] = want_grad ? res[3 + p] : 0.0;
  if (nbad <= -2) {
    out[0] = HUGE_VAL;
    return set_error(GOO_ERR_RANGE, "%.0f events in [%lld, %lld) lie outside the observable limits", -nbad - 2,
                     (long long)begin, (long long)end);
  }
  if (nbad < 0) {
    out[0] = HUGE_VAL;
    return set_error(GOO_ERR_TIMEOUT, "a device wait for event data gave up in [%lld, %lld)", (long long)begin,
                     (long long)end);
  }
  if (nbad > 0) {
    out[0] = HUGE_VAL;
    return set_error(GOO_ERR_NONPOSITIVE_PDF, "density is <= 0 for %.0f events in [%lld, %lld)", nbad,
                     (long long)begin, (long long)end);
  }
  return GOO_OK;
}

int goo_gram(goo_model* m, const double* theta, int precision, double* out, int* K_out) {
  if (!m || !out || !K_out) return set_error(GOO_ERR_ARG, "goo_gram: NULL argument");
  if (m->kind != 1 && m->kind != 2) return set_error(GOO_ERR_STATE, "goo_gram: not an amplitude model");
  if (precision != GOO_F64 && precision != GOO_F32) return set_error(GOO_ERR_ARG, "precision=%d", precision);
  GOO_TRY(check_theta(m, theta));
  GOO_CUDA_TRY(cudaSetDevice(m->ctx->device));
  if (m->kind == 2) return td4_gram(m, precision, out, K_out);
  return dalitz_gram(m, theta, precision, out, K_out);
}

int goo_model_set_lineshapes(goo_model* m, int mode) {
  if (!m) return set_error(GOO_ERR_ARG, "goo_model_set_lineshapes: NULL model");
  if (m->kind != 1) return set_error(GOO_ERR_UNSUPPORTED, "goo_model_set_lineshapes: not a three-body amplitude model");
  return dalitz_set_lineshapes(m, mode);
}

int goo_model_set_coefficients(goo_model* m, int form) {
  if (!m) return set_error(GOO_ERR_ARG, "goo_model_set_coefficients: NULL model");
  if (m->kind != 1) return set_error(GOO_ERR_UNSUPPORTED, "goo_model_set_coefficients: not a three-body amplitude model");
  return dalitz_set_coefficients(m, form);
}

int goo_model_set_jit(goo_model* m, int mode) {
  if (!m) return set_error(GOO_ERR_ARG, "goo_model_set_jit: NULL model");
  if (mode != 0 && mode != 1) return set_error(GOO_ERR_ARG, "goo_model_set_jit: mode=%d", mode);
  m->jit_mode = mode;
  m->jit_status = mode;
  m->ev2_fn[0] = m->ev2_fn[1] = m->ev2_fn[2] = m->ev2_fn[3] = nullptr;
  return GOO_OK;
}

int goo_model_jit_status(const goo_model* m) { return m ? m->jit_status : GOO_ERR_ARG; }

int goo_amplitude_cache(goo_model* m, const goo_dataset* ds, const double* theta, int precision, const void** dev_ptr,
                        int* n_amp) {
  if (!m || !ds || !dev_ptr || !n_amp) return set_error(GOO_ERR_ARG, "goo_amplitude_cache: NULL argument");
  if (m->kind != 1 && m->kind != 2) return set_error(GOO_ERR_STATE, "goo_amplitude_cache: not an amplitude model");
  GOO_TRY(check_model_dataset(m, ds, precision));
  GOO_TRY(check_theta(m, theta));
  GOO_CUDA_TRY(cudaSetDevice(m->ctx->device));
  if (m->kind == 2) return td4_amplitudes(m, ds, precision, dev_ptr, n_amp);
  return dalitz_amplitudes(m, ds, theta, precision, dev_ptr, n_amp);
}

}  // extern "C"
