// model.cuh -- device-side layout of a flattened sum-of-products model and the library's
// model object.
#pragma once

#include "common.cuh"

namespace goo {

constexpr int kMaxAdd = 8;

struct LeafDev {
  int op, col;
  int par[3];          // parameter indices (-1: unused)
  int pad;
  float f[6];          // FP32 constants (offsets as hi/lo pairs)
  double d[6];         // FP64 constants
  double a_ref;        // grid reference exponent of this leaf (upper bound of a over its range)
  float a_ref_hi, a_ref_lo;
};

struct CompDev {
  int n_leaf, n_fac;
  int fac_add[8], fac_pos[8];      // weight = product of ADD factors (add index, child position)
  float off_hi, off_lo;            // -log N_k as float hi + lo
  float w_hi, w_lo;                // w_k as float hi + lo
  float a_ref_hi, a_ref_lo;        // grid reference exponent
  double w, log_norm, a_ref;
};

struct AddDev {
  int n_child;
  int frac[GOO_MAX_CHILD];
};

struct GridDev {
  int ndim;
  int bins[kMaxObs];
  int dim_of_col[kMaxObs];         // grid dimension of each observable (-1: not used)
  float h_hi[kMaxObs], h_lo[kMaxObs], lo_hi[kMaxObs], lo_lo[kMaxObs];
  double h64[kMaxObs], lo64[kMaxObs];
  double cell_volume;
};

struct ModelDev {
  int nK, n_obs, n_params, norm_kind, n_add;
  int grid_separable;                  // GRID: every product's leaves on distinct observables
  double lo[kMaxObs], hi[kMaxObs];
  CompDev comp[kMaxComp];
  LeafDev leaf[kMaxComp * kMaxLeaf];   // leaf l of product k at [k * kMaxLeaf + l]
  AddDev add[kMaxAdd];
  GridDev grid[kMaxComp];
  double dw[kMaxComp][kMaxParams];     // d w_k / d theta_p
  double dlogN[kMaxComp][kMaxParams];  // d log N_k / d theta_p
};

#ifndef __CUDACC_RTC__
struct DalitzModel;  // three-body amplitude models (dalitz.cu)
struct Td4Model;     // time-dependent four-body models (td4.cu)

int build_sop_model(goo_ctx* ctx, const goo_node* nodes, int n_nodes, int n_params, int n_obs,
                    const double* lo, const double* hi, goo_model* m);
int sop_set_norm(goo_model* m, const goo_norm_spec* spec);
// Uploads the prepared model block and launches the grid normalisation, unless norm_in_event
// (sop_norm_in_event true, and the following sop_events call passes it too).
int sop_prepare(goo_model* m, const double* theta_host, int precision, bool norm_in_event = false);
// True when the FP32 event kernel for this model normalises a separable grid itself.
bool sop_norm_in_event(const goo_model* m, int precision, bool grad);
void host_prep(ModelDev& h, const double* theta, int precision);
// result: the record's destination (kResultDoubles + 1 doubles; null: the context's device
// scratch record); the kernel writes each field once and sets its completion word
// (kResultFlag) last.
int sop_events(goo_model* m, const goo_dataset* ds, int64_t begin, int64_t end, int precision, bool grad,
               int out_mode, bool norm_in_event = false, double* result = nullptr);
int sop_eval_logf(goo_model* m, const goo_dataset* ds, int precision, double* logf_dev);

int build_dalitz_model(goo_ctx* ctx, const goo_node* nodes, int n_nodes, int n_params, int n_obs,
                       const double* lo, const double* hi, goo_model* m);
int dalitz_set_norm(goo_model* m, const goo_norm_spec* spec);
void dalitz_free(goo_model* m);
int dalitz_normalise(goo_model* m, const double* theta, int precision, double* norm_out);
int dalitz_nll(goo_model* m, const goo_dataset* ds, int64_t begin, int64_t end, const double* theta,
               int precision, bool grad, double* out, int out_mode);
int dalitz_eval_logf(goo_model* m, const goo_dataset* ds, const double* theta, int precision, double* logf_dev);
int dalitz_gram(goo_model* m, const double* theta, int precision, double* out, int* K_out);
int dalitz_amplitudes(goo_model* m, const goo_dataset* ds, const double* theta, int precision, const void** cache,
                      int* nbw);
int dalitz_set_lineshapes(goo_model* m, int mode);
bool dalitz_lineshape_param(const goo_model* m, int p);  // p is a resonance mass or width
bool dalitz_floating(const goo_model* m);
bool dalitz_time_dependent(const goo_model* m);
int dalitz_set_coefficients(goo_model* m, int form);

int build_td4_model(goo_ctx* ctx, const goo_node* nodes, int n_nodes, int n_params, int n_obs, goo_model* m);
int td4_set_norm(goo_model* m, const goo_norm_spec* spec);
void td4_free(goo_model* m);
int td4_normalise(goo_model* m, const double* theta, int precision, double* norm_out);
int td4_nll(goo_model* m, const goo_dataset* ds, int64_t begin, int64_t end, const double* theta, int precision,
            bool grad, double* out, int out_mode);
int td4_eval_logf(goo_model* m, const goo_dataset* ds, const double* theta, int precision, double* logf_dev);
int td4_gram(goo_model* m, int precision, double* out, int* K_out);
int td4_amplitudes(goo_model* m, const goo_dataset* ds, int precision, const void** cache, int* n_amp);

}  // namespace goo

struct goo_model {
  goo_ctx* ctx = nullptr;
  int kind = 0;  // 0: sum of products, 1: coherent amplitude sum, 2: time-dependent four-body
  int n_params = 0, n_obs = 0;
  double lo[goo::kMaxCols] = {};
  double hi[goo::kMaxCols] = {};
  goo_norm_spec norm{};
  int max_leaf = 0;
  goo::ModelDev host{};
  goo::ModelDev* dev = nullptr;
  goo::ModelDev* stage = nullptr;  // pinned host staging of the per-call model block
  goo::DalitzModel* dalitz = nullptr;
  goo::Td4Model* td4 = nullptr;
  bool counted = false;  // included in ctx->live
  // FP32 packed-pair kernel specialised for this model at run time (goo_model_set_jit):
  // jit_mode 1 (default) or 0; jit_status as goo_model_jit_status reports it
  int jit_mode = 1;
  int jit_status = 1;
  // the packed-pair event kernel resolved for this model (index: gradient form) and the
  // jit_status it came with; reset by goo_model_set_jit
  // the pair kernel per gradient form (index gi) and column source (+2: host columns read
  // directly), resolved on first use
  const void* ev2_fn[4] = {nullptr, nullptr, nullptr, nullptr};
  int ev2_status[4] = {0, 0, 0, 0};
};

namespace goo {
// What the toy-MC server needs from an amplitude model (dalitz.cu): device lineshape
// constants and FP32-path Gram matrix at theta, amplitude/parameter layout and the box.
struct AmpModelInfo {
  const void* dalitz_dev;   // DalitzDev*
  const double* gram_dev;   // K x K complex, FP64 (from the float32 MC cache)
  int K, nbw, has_nr;
  int par_re[16], par_im[16];
  double lo12, hi12, lo13, hi13;
  double M, m1, m2, m3;
};
int dalitz_server_info(goo_model* m, const double* theta, AmpModelInfo* info);
}  // namespace goo
#else
}  // namespace goo
#endif  // __CUDACC_RTC__
