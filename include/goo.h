/*
 * goo.h -- C ABI of the GB300 unbinned-likelihood engine.
 *
 * The engine evaluates a composite probability density f(x; theta) at every event of
 * an unbinned, structure-of-arrays dataset, normalises it (closed form, midpoint grid
 * or Monte-Carlo phase-space sample) and reduces the negative log-likelihood
 *     NLL(theta) = - sum_i log f(x_i; theta)
 * and its gradient with respect to theta in hand-written sm_103a kernels.
 *
 * Paper: GooFit 2.0 (arXiv:1710.08826).  The paper's user model is Variables
 * (observables and parameters) feeding PDFs, combination PDFs that combine them, and a
 * FitManager that fits the final PDF to a binned or unbinned DataSet (Fig. 1); the
 * time of a fit is dominated by evaluating the function independently at every data
 * point (Sec. 1).  Each call below cites the passage it restates.
 *
 * Conventions for every call:
 *   - Return value: GOO_OK (0) or a negative GOO_ERR_* code.  No C++ exception crosses
 *     this boundary.  goo_last_error() returns a thread-local message for the last
 *     failing call on the calling thread.
 *   - "host" pointers are CPU memory owned by the caller; "device" pointers are CUDA
 *     global memory on the context's device.  Output pointers are host memory unless
 *     stated otherwise, and every call is synchronous with respect to its host outputs.
 *   - theta is a host array of n_params doubles in the order of the model's parameter
 *     indices.  Gradients are returned for all n_params entries.
 *   - Objects (goo_ctx, goo_dataset, goo_model) are owned by the library and released
 *     with the matching *_free / goo_finalize call.  A dataset or model must not outlive
 *     its context.  Calls on one context must not run concurrently from several threads.
 */
#ifndef GOO_H
#define GOO_H

#ifdef __CUDACC_RTC__
/* device code compiled at run time (NVRTC) sees the enums only; the integer types come
   from the compiler's own headers */
#include <cuda/std/cstdint>
typedef cuda::std::int32_t int32_t;
typedef cuda::std::int64_t int64_t;
typedef cuda::std::uint64_t uint64_t;
typedef cuda::std::uint32_t uint32_t;
typedef cuda::std::uintptr_t uintptr_t;
#else
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
enum {
  GOO_OK = 0,
  GOO_ERR_ARG = -1,             /* invalid argument (null pointer, bad size, bad node)     */
  GOO_ERR_RANGE = -2,           /* event outside its observable's [lo, hi] at upload       */
  GOO_ERR_CUDA = -3,            /* a CUDA runtime call failed                               */
  GOO_ERR_OOM = -4,             /* device allocation failed or an admission budget is full  */
  GOO_ERR_NONPOSITIVE_PDF = -5, /* f(x_i) <= 0 for some event: the NLL is +inf              */
  GOO_ERR_TIMEOUT = -6,         /* a bounded device wait gave up                            */
  GOO_ERR_STATE = -7,           /* call not valid in the object's current state            */
  GOO_ERR_UNSUPPORTED = -8      /* model/normalisation combination not implemented          */
};

/* ---- precisions / column types ----------------------------------------------------- */
enum {
  GOO_F64 = 0, /* float64 columns; plain FP64 evaluation and accumulation                  */
  GOO_F32 = 1  /* float32 columns; FP32 per-event evaluation, compensated FP32/double-float
                  accumulation, FP64 final combination                                    */
};

/* ---- dataset upload flags ----------------------------------------------------------- */
enum {
  GOO_COPY = 0,         /* cols are host pointers; the library copies them                 */
  GOO_BORROW_DEVICE = 1, /* cols are device pointers that must outlive the dataset        */
  GOO_COPY_MAPPED = 2,  /* cols are pinned host pointers (cudaHostAlloc / registered); the
                           ingest kernel reads them over the host link itself, with no
                           separate copy-engine transfer                                   */
  GOO_BORROW_HOST = 3   /* cols are pinned, device-mapped float32 host arrays kept by
                           reference: nothing is copied, every evaluation reads them over the
                           host link and range-checks them (see goo_dataset_upload)        */
};

/* ---- model nodes --------------------------------------------------------------------- */
enum {
  GOO_OP_GAUSS = 1,  /* par[0]=mu, par[1]=sigma          exp(-(x-mu)^2/(2 sigma^2))           */
  GOO_OP_EXPO = 2,   /* par[0]=lambda                     exp(lambda x)                        */
  GOO_OP_POLY2 = 3,  /* par[0]=a1, par[1]=a2              1 + a1 x + a2 x^2                    */
  GOO_OP_ARGUS = 4,  /* par[0]=m0, par[1]=c, par[2]=p     m (1-m^2/m0^2)^p exp(c(1-m^2/m0^2)) */
  GOO_OP_PROD = 10,  /* product of the children (children on disjoint observables)        */
  GOO_OP_ADD = 11,   /* sum_k w_k child_k / norm(child_k); par[0..K-2] = fractions,
                        w_{K-1} = 1 - sum of the fractions                                 */
  GOO_OP_BW = 20,    /* Breit-Wigner amplitude: par[0]=m0, par[1]=width, par[2]=Re c,
                        par[3]=Im c; ival[0]=spin (0..2), ival[1]=pair (0:12, 1:13, 2:23) */
  GOO_OP_NR = 21,    /* constant (non-resonant) amplitude: par[2]=Re c, par[3]=Im c       */
  GOO_OP_COHERENT = 22, /* |sum_k c_k A_k|^2 over its BW/NR children; obs[0]=s12, obs[1]=s13;
                          dval = {M, m1, m2, m3, r_res, r_parent}                          */
  /* Time-dependent four-body amplitude model (paper Sec. 5: time-dependent amplitude
   * analysis of four-body decays for a mixing measurement).  The model's observables are,
   * in this order, m12, m34, cos th12, cos th34, phi, t (six dataset columns).
   *   A = sum_k c_k a_k (free coefficients), B = sum_k b_k a_k (fixed coefficients),
   *   rate R = e^{-G t}[(|A|^2+|B|^2)/2 cosh(yGt) + (|A|^2-|B|^2)/2 cos(xGt)
   *            + Re(AB*) sinh(yGt) + Im(AB*) sin(xGt)] (G = 1/tau) convolved with a Gaussian
   *   of width sigma_t; normalised over phase space (MC Gram matrix) and all t.          */
  GOO_OP_TD4 = 23,   /* root over GOO_OP_AMP4 children: par[0]=x, par[1]=y, par[2]=tau (ps),
                        par[3]=sigma_t (ps); dval = {M, m1, m2, m3, m4, r (barrier radius)}  */
  GOO_OP_AMP4 = 24,  /* a_k = F(m12; dval[0]=m0, dval[1]=width) F(m34; dval[2]=m0,
                        dval[3]=width) W(cos th12, cos th34, phi), F a Breit-Wigner with
                        running width and Blatt-Weisskopf factors of the spins that
                        ival[0] = GOO_ANG_* fixes; par[0]=Re c_k, par[1]=Im c_k (free),
                        dval[4]=Re b_k, dval[5]=Im b_k (fixed)                          */
  /* Time-dependent three-body amplitude model (paper Sec. 5 and Table 2: a time-dependent
   * amplitude analysis of D0 -> pi+ pi- pi0).  Particle 1 is the neutral, 2 and 3 the
   * CP-conjugate pair (m2 = m3); observables s12, s13 and t.  The anti-particle's amplitudes
   * are the same lineshapes at the exchanged point, abar_k(s12, s13) = a_k(s13, s12), and
   * A = sum_k c_k a_k, B = sum_k c_k abar_k (no CP violation, q/p = 1).  The rate and its
   * normalisation are GOO_OP_TD4's with these A and B; the normalisation uses three MC Gram
   * matrices <a_k a_l*>, <abar_k abar_l*>, <a_k abar_l*>. */
  GOO_OP_TD3 = 25    /* root over GOO_OP_BW / GOO_OP_NR children (as GOO_OP_COHERENT):
                        obs[0]=s12, obs[1]=s13, ival[0]=t; par[0..3] = x, y, tau (ps),
                        sigma_t (ps); dval = {M, m1, m2, m3, r_res, r_parent}            */
};

/* Angular structures of GOO_OP_AMP4 (spins of the 12 and 34 resonances in brackets; s = sin):
 * SS (0,0) 1; VS0 (1,0) cos th12; SV0 (0,1) cos th34; VV0 (1,1) cos th12 cos th34;
 * VVPAR (1,1) s12 s34 cos phi; VVPERP (1,1) i s12 s34 sin phi; TS0 (2,0) P2(cos th12);
 * TV0 (2,1) P2(cos th12) cos th34, with P2(c) = (3c^2 - 1)/2. */
enum {
  GOO_ANG_SS = 0, GOO_ANG_VS0 = 1, GOO_ANG_SV0 = 2, GOO_ANG_VV0 = 3, GOO_ANG_VVPAR = 4, GOO_ANG_VVPERP = 5,
  GOO_ANG_TS0 = 6, GOO_ANG_TV0 = 7
};

#define GOO_MAX_CHILD 16

/* One node of the model's expression tree.  Nodes are given in post-order: every child
 * index is smaller than its parent's, and the last node is the root.  Unused par[] and
 * obs[] slots are -1.  Paper: basic PDFs, combination PDFs and amplitude PDFs
 * (Fig. 1; Sec. 1). */
typedef struct goo_node {
  int32_t op;
  int32_t obs[2];                 /* observable (dataset column) indices                  */
  int32_t par[8];                 /* parameter indices into theta                         */
  int32_t n_child;
  int32_t child[GOO_MAX_CHILD];   /* indices of the child nodes                           */
  int32_t ival[2];                /* integer attributes (GOO_OP_BW)                        */
  double dval[6];                 /* real attributes (GOO_OP_COHERENT)                     */
} goo_node;

/* ---- normalisation ------------------------------------------------------------------- */
enum {
  GOO_NORM_ANALYTIC = 0, /* closed-form integrals of the leaves over the observable ranges */
  GOO_NORM_GRID = 1,     /* midpoint rule per normalised component, bins[] per observable  */
  GOO_NORM_MC = 2        /* mean over a phase-space MC dataset (amplitude models): the Gram
                            matrix <a_k a_l*>; the t column of a GOO_OP_TD4 MC is ignored */
};

typedef struct goo_dataset goo_dataset;

typedef struct goo_norm_spec {
  int32_t kind;            /* GOO_NORM_*                                                  */
  int32_t bins[4];         /* GRID: number of bins of observable 0..3                    */
  const goo_dataset* mc;   /* MC: phase-space sample; borrowed, must outlive the model   */
} goo_norm_spec;

typedef struct goo_ctx goo_ctx;
typedef struct goo_model goo_model;

/* ---- context ------------------------------------------------------------------------- */
/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t (for example
 * torch.cuda.current_stream().cuda_stream) or NULL for a stream the library creates.
 * All work of the context is ordered on that stream. */
int goo_init(int device, void* cuda_stream, goo_ctx** out);
/* goo_finalize fails with GOO_ERR_STATE (and frees nothing) while datasets, models or servers
 * created on ctx are still alive: free them first. */
int goo_finalize(goo_ctx* ctx);
const char* goo_last_error(void);
/* Library version string and the number of kernel launches issued so far by ctx. */
const char* goo_version(void);
int64_t goo_launch_count(const goo_ctx* ctx);
/* Per-kernel timing statistics (paper Sec. 3: fits report timing statistics).
 * When enabled, every kernel launch of ctx is bracketed by CUDA events on ctx's stream.
 * goo_timing_read folds finished launches into per-kernel totals and copies up to
 * max_entries of them: names (64 chars each, NUL-terminated), launch counts and total
 * milliseconds; it returns the number of kernels with statistics (or a negative code),
 * and clears the table when reset != 0.  It waits for the recorded launches to finish. */
int goo_timing_enable(goo_ctx* ctx, int on);
int goo_timing_read(goo_ctx* ctx, int max_entries, char* names, int64_t* counts, double* total_ms, int reset);
/* Limit of the kernels' bounded waits.  The paper describes no failure handling; this call
 * serves the library's own failure detection.  Kernels that stage their input tiles in
 * shared memory by bulk copies wait for each tile on an mbarrier for at most `cycles` SM
 * clocks (0 restores the default of 2e9 clocks, about one second at 2 GHz; at most
 * 2^32 - 1).  A wait that runs out makes the evaluation return GOO_ERR_TIMEOUT (nll = +inf)
 * while the context stays usable; before a block exits it always waits up to the default
 * limit for its own copies still in flight.  A very small limit therefore turns evaluations
 * whose copies have not landed in time into GOO_ERR_TIMEOUT without a fault, which is how
 * the timeout path is tested.  The setting applies to every later call on ctx (evaluations,
 * fits, servers); it is ordered on ctx's stream and the call returns once it is in place.
 * GOO_ERR_ARG for a NULL context or a limit out of range. */
int goo_set_wait_limit(goo_ctx* ctx, int64_t cycles);
/* Failure-detection test hook (the paper describes no failure handling).  With tile >= 0 the
 * first block of the staged FP32 kernels of the sum-of-products and three-body models does
 * not issue the copies of its tile number `tile` (counted in the block's own order), so the
 * waits for that tile run out after the wait limit and the evaluation returns
 * GOO_ERR_TIMEOUT; nothing faults, and the block drains the copies it did issue before it
 * exits.  tile = -1 clears the hook.  Ordered on ctx's stream; applies to later calls on ctx.
 * Set a short wait limit first (goo_set_wait_limit), or each such evaluation waits about a
 * second.  GOO_ERR_ARG for a NULL context or tile < -1. */
int goo_debug_withhold_tile(goo_ctx* ctx, int64_t tile);

/* ---- data (paper: DataSet, Fig. 1 and Sec. 4) ------------------------------------------------
 * Upload `ncols` (1..8) structure-of-arrays columns of n_events values each, of type `dtype`
 * (GOO_F64 or GOO_F32).  With GOO_COPY the columns are host arrays copied to the device;
 * with GOO_BORROW_DEVICE they are device arrays (16-byte aligned) kept by reference.
 * lo[c], hi[c] are the limits of observable c.  Every event is range-checked on the device
 * (Sec. 4: data loaded outside the observables' ranges is caught at run time): if
 * any value lies outside its [lo, hi] (or is NaN) the call fails with GOO_ERR_RANGE, no
 * dataset is created, and *n_bad (if not NULL) receives the number of offending events.
 * The device keeps both a float64 and a float32 copy of every column, written by one fused
 * conversion and range-check pass.  GOO_COPY_MAPPED fails with GOO_ERR_ARG unless every
 * column is pinned host memory.
 *
 * GOO_BORROW_HOST (dtype GOO_F32 only) keeps pinned, device-mapped host columns by reference
 * (16-byte aligned; they must outlive the dataset) and copies nothing: the caller may rewrite
 * their contents between evaluations (with no evaluation in flight).  Every FP32 evaluation of
 * a sum-of-product model reads the events over the host link inside its event kernel, the
 * transfer overlapped with the arithmetic, and checks each event against the limits: an
 * evaluation that meets events outside them (or NaN) fails with GOO_ERR_RANGE.  The upload
 * itself checks nothing.  Such a dataset serves goo_nll / goo_nll_grad / goo_nll_partial in
 * GOO_F32 with sum-of-product models of at most 2 products of 3 leaves (or, without the
 * gradient, 4 of 4) and no weights; anything else (FP64 evaluation, amplitude models,
 * goo_dataset_update, goo_dataset_set_weights, goo_dataset_column in GOO_F64) fails with
 * GOO_ERR_UNSUPPORTED or GOO_ERR_STATE. */
int goo_dataset_upload(goo_ctx* ctx, int ncols, const void* const* cols, int dtype,
                       int64_t n_events, const double* lo, const double* hi, int flags,
                       goo_dataset** out, int64_t* n_bad);
int goo_dataset_free(goo_dataset* ds);
/* Replace the events of a dataset created with GOO_COPY or GOO_COPY_MAPPED by n_events new
 * ones (0 <= n_events <= the count it was created with), reusing its device buffers: the
 * streaming form of goo_dataset_upload for a new batch of events each step.  cols: one host
 * array per column (the dataset's ncols, the same limits), flags GOO_COPY or GOO_COPY_MAPPED
 * as for the upload.  Waits for the launches in flight, then copies, converts and
 * range-checks like the upload.  Weights are removed and amplitude caches and MC Gram
 * matrices built from the old events are invalidated.  Errors: GOO_ERR_STATE for a dataset
 * that borrows its columns, GOO_ERR_ARG for a bad size or flag, GOO_ERR_RANGE (with
 * *n_bad) when events lie outside the limits, after which the dataset holds no events. */
int goo_dataset_update(goo_dataset* ds, const void* const* cols, int dtype, int64_t n_events, int flags,
                       int64_t* n_bad);
int64_t goo_dataset_size(const goo_dataset* ds);
/* Device pointer of column `col` in the given precision (for zero-copy consumers). */
const void* goo_dataset_column(const goo_dataset* ds, int col, int dtype);
/* Per-event weights w[0..n_events) (paper: binned data sets, Fig. 1 and Sec. 4).  A binned
 * dataset is uploaded as one event per bin (its centre) and weighted by the bin's count;
 * the NLL of a sum-of-product model is then -sum_i w_i log f(x_i) (the multinomial
 * likelihood of the bin contents with f at the bin centres, up to a theta-independent
 * constant) and its gradient is weighted the same way; events of weight 0 (empty bins) are
 * skipped.  Weights must be finite and >= 0 (else GOO_ERR_ARG, nothing changed).  The host
 * array is copied (the caller keeps it); w = NULL removes the weights.  Amplitude models and
 * goo_nll_grad_batch refuse a weighted dataset with GOO_ERR_UNSUPPORTED; goo_eval_logf
 * ignores the weights; goo_nll_partial's third record entry stays the event count. */
int goo_dataset_set_weights(goo_dataset* ds, const double* w);

/* ---- model (paper: PDFs and combination PDFs, Fig. 1 and Sec. 1) -----------------------------
 * Build a model from `n_nodes` post-order nodes over `n_params` parameters and `n_obs`
 * observables with limits obs_lo/obs_hi (the normalisation range).  Sum/product trees are
 * flattened to a sum of products of leaves (at most 4 products of at most 4 leaves after
 * flattening) over at most 4 observables; a GOO_OP_COHERENT root builds a three-body
 * amplitude model and a GOO_OP_TD4 root the time-dependent four-body model (6 observables;
 * at most 8 for any model).  The default normalisation is GOO_NORM_ANALYTIC for sum/product
 * trees; amplitude models need GOO_NORM_MC. */
int goo_model_build(goo_ctx* ctx, const goo_node* nodes, int n_nodes, int n_params, int n_obs,
                    const double* obs_lo, const double* obs_hi, goo_model** out);
int goo_model_set_norm(goo_model* model, const goo_norm_spec* spec);
int goo_model_free(goo_model* model);
/* Number of normalised components (products) of the flattened model. */
int goo_model_components(const goo_model* model);

/* ---- normalisation (a5) ---------------------------------------------------------------------
 * Integral of each normalised component at theta, in `precision`; norms_out receives
 * goo_model_components() doubles (for amplitude models one value: the MC mean of |S|^2, or
 * for GOO_OP_TD4 the MC mean of the rate integrated over all t). */
int goo_normalise(goo_model* model, const double* theta, int precision, double* norms_out);

/* ---- likelihood (a1-a7; paper Sec. 1: the per-event evaluation dominates a fit) -------------- */
int goo_nll(goo_model* model, const goo_dataset* ds, const double* theta, int precision,
            double* nll_out);
/* NLL and its gradient d NLL / d theta (hand-written adjoint).  grad_out: n_params doubles. */
int goo_nll_grad(goo_model* model, const goo_dataset* ds, const double* theta, int precision,
                 double* nll_out, double* grad_out);
/* Per-event log f(x_i; theta) written to the device array logf_dev (n_events doubles). */
int goo_eval_logf(goo_model* model, const goo_dataset* ds, const double* theta, int precision,
                  double* logf_dev);

/* ---- amplitude models (paper Sec. 1, Sec. 4, Sec. 5) ------------------------------------------
 * For a GOO_OP_COHERENT model: the MC Gram matrix G_kl = mean over the MC sample of
 * A_k conj(A_l) at theta's lineshape parameters (K x K complex, row-major, re/im interleaved,
 * amplitudes in tree order with the non-resonant amplitude last), K written to *K_out; and
 * the device pointer of the dataset's cached resonance amplitudes (built if stale; layout:
 * GOO_F32 -> ceil(n_amp/2) planes of float4 (re_k, im_k, re_k+1, im_k+1) per event,
 * GOO_F64 -> n_amp planes of double2 per event; plane p starts at p * n_events).  The cache
 * is owned by the dataset and rebuilt when the model or its lineshape parameters change
 * (paper Sec. 4: cached partial results in structure-of-arrays form, change detection). */
int goo_gram(goo_model* model, const double* theta, int precision, double* out, int* K_out);
int goo_amplitude_cache(goo_model* model, const goo_dataset* ds, const double* theta, int precision,
                        const void** dev_ptr, int* n_amp);
/* Lineshape handling of a GOO_OP_COHERENT model (paper Sec. 4: cached lineshapes, recomputed
 * when their parameters change).
 *   GOO_LINESHAPE_CACHED (default): the amplitude cache and the MC Gram matrix hold the
 *     lineshapes; the NLL is exact at any theta, but goo_nll_grad returns 0 for the
 *     resonance masses and widths (constants of the cache), and goo_fit refuses to free them
 *     with the adjoint gradient.
 *   GOO_LINESHAPE_FLOATING: goo_nll / goo_nll_grad / goo_nll_partial evaluate every
 *     Breit-Wigner amplitude per event and per MC point on each call (no cache, no Gram
 *     matrix), with d A / d m0 and d A / d Gamma0 from the lineshape formula, so the gradient
 *     covers every parameter; N is the MC mean of |S|^2 at theta.  goo_normalise,
 *     goo_eval_logf and goo_gram keep using the cache.
 * GOO_ERR_UNSUPPORTED for other models, GOO_ERR_ARG for another mode. */
enum { GOO_LINESHAPE_CACHED = 0, GOO_LINESHAPE_FLOATING = 1 };
int goo_model_set_lineshapes(goo_model* model, int mode);
/* Coefficient form of a GOO_OP_COHERENT or GOO_OP_TD3 model's amplitudes (the paper's
 * amplitude PDFs take complex coefficients; the polar form is the usual alternative).  With
 * GOO_COEF_POLAR the two coefficient parameters of an amplitude (par[2], par[3]) are its
 * magnitude r and phase phi (radians): c = r e^{i phi}; goo_nll_grad then returns d/dr and
 * d/dphi.  GOO_COEF_CARTESIAN (default): (Re c, Im c).  The toy server takes Cartesian models
 * only.  GOO_ERR_UNSUPPORTED for other models, GOO_ERR_ARG for another form. */
enum { GOO_COEF_CARTESIAN = 0, GOO_COEF_POLAR = 1 };
int goo_model_set_coefficients(goo_model* model, int form);
/* Run-time kernel specialisation of a sum-of-products model's FP32 evaluation.  With mode 1
 * (the default) the first FP32 evaluation that runs in the packed-pair event kernel compiles
 * that kernel for the model's leaf signature with NVRTC (a second or so, once per signature
 * and process); later evaluations launch the compiled kernel.  Mode 0 keeps the interpreter
 * compiled into the library.  Both compute the same sums; they may differ in the last bits
 * through fused multiply-adds.  GOO_ERR_ARG for another mode.
 * goo_model_jit_status: 0 off, 1 on and not yet used, 2 the last FP32 evaluation ran the
 * specialised kernel, -1 compilation failed and the interpreter ran instead. */
int goo_model_set_jit(goo_model* model, int mode);
int goo_model_jit_status(const goo_model* model);
/* Compile the packed-pair event kernel for a K x L slot shape (K products of at most L
 * leaves; 1 <= K, L <= 4), with or without gradient lanes, for a leaf signature (4 bits per
 * slot k * L + l: the leaf's GOO_OP_* code, 0 for an empty slot) and column map (2 bits per
 * slot: the leaf's observable), as goo_model_set_jit does on a model's first evaluation,
 * without loading it: needs no GPU.  For checking NVRTC and the kernel sources on a machine
 * before the first evaluation.  *cubin_bytes (if not NULL) receives the image size.
 * GOO_ERR_CUDA with NVRTC's log in goo_last_error on failure. */
int goo_jit_check(int K, int L, int grad, unsigned long long sig, unsigned long long cols, int64_t* cubin_bytes);

/* ---- fitting (paper: the FitManager, Fig. 1; Minuit 2 as the default minimiser, Sec. 4) -------
 * Minimises the NLL of `model` on `ds` over the parameters with free_mask[p] != 0, starting
 * from theta (host, n_params doubles), which receives the minimum.  scale[p] > 0 is a typical
 * step of each free parameter (the minimiser works in units of it).  Quasi-Newton BFGS with a
 * backtracking line search, then (polish != 0) Newton steps on a finite-difference Hessian
 * of the gradient; errors_out (NULL or n_params doubles) receives sqrt(diag(H^-1)) for free
 * parameters and 0 for fixed ones.  The gradient is the adjoint kernel (GOO_GRAD_ADJOINT) or
 * central differences of goo_nll (GOO_GRAD_FD, the plain path).  With refine != 0, an FP32
 * fit (adjoint gradient, polish on) ends in FP64: after BFGS on FP32 evaluations, Newton steps
 * use FP64 adjoint gradients with the finite-difference Hessian (from FP32 gradients when that
 * Hessian is positive definite, else from FP64 ones), so that the minimum is the FP64
 * likelihood's at a small cost; res->nll is then the FP64 NLL.  res->status: 0 converged
 * (0 <= EDM = g^T H^-1 g / 2 < edm_tol), 1 iteration limit, 2 line-search failure, 3 the
 * Hessian at the end is not positive definite.  Returns an error code only for invalid
 * arguments or a non-finite NLL at the start. */
enum { GOO_GRAD_ADJOINT = 0, GOO_GRAD_FD = 1 };
typedef struct goo_fit_options {
  int32_t precision;  /* GOO_F64 or GOO_F32                                                 */
  int32_t gradient;   /* GOO_GRAD_ADJOINT or GOO_GRAD_FD                                    */
  int32_t max_iter;   /* BFGS iterations (<= 0: 500)                                        */
  int32_t polish;     /* Newton steps on the finite-difference Hessian after BFGS           */
  double edm_tol;     /* convergence threshold on EDM (<= 0: 1e-6)                          */
  int32_t refine;     /* FP32 fits: final Newton steps on FP64 gradients (see above)        */
} goo_fit_options;
typedef struct goo_fit_result {
  double nll, edm, wall_ms;
  int32_t iterations, nll_evals, grad_evals, status;
} goo_fit_result;
int goo_fit(goo_model* model, const goo_dataset* ds, double* theta, const int* free_mask, const double* scale,
            const goo_fit_options* options, double* errors_out, goo_fit_result* res);

/* ---- toy-MC fits served with continuous batching (paper Sec. 5: toy MC generation; Fig. 1) ----
 * For an amplitude model with a non-resonant reference amplitude, <= 8 resonances, fixed
 * lineshapes and an MC normalisation sample.  A request is one pseudo-experiment: n_events
 * generated on the device from the model at theta_gen (Philox4x64-10 streams keyed by `seed`,
 * accept-reject against the cell envelope below; the toy is the first n accepted candidates
 * in candidate order), then fitted from theta_start (NULL: theta_gen) over the resonance
 * coefficients (free_mask must mark exactly those).  Requests are admitted in submission
 * order while a fit slot and 72 bytes per event of the device arena are free.  Each
 * goo_server_step admits and generates new fits, runs ONE batched NLL+gradient launch over
 * every active fit (fixed per-fit tiles, per-fit reduction in tile order: a fit's result
 * does not depend on the other fits in the batch) and ONE launch advancing every fit's
 * device-resident minimiser (BFGS, then Newton steps on a finite-difference Hessian whose
 * inverse gives the errors), then retires finished fits.  goo_server_result returns
 * GOO_ERR_STATE until the fit is finished.  stats: see goo_server_stats. */
typedef struct goo_server goo_server;
/* Envelope of the toy generator: an n12 x n13 grid of equal cells over the Dalitz box
 * [(m1+m2)^2, (M-m3)^2] x [(m1+m3)^2, (M-m2)^2], cell (i, j) at index i * n13 + j, with
 * bound[c] >= |S|^2 at every point of cell c inside the kinematic region.  Candidate j of a
 * toy with seed s uses the Philox4x64-10 words w0..w3 at counter (j, 0, 0, 0), key
 * (s, 0x6f6f67): the cell is the first c with (w0 >> 32) < thr[c], thr[c] =
 * floor(S_c / W * 2^32) (S_c the FP64 sum of bound[0..c], W the total; thr[last] = 2^32);
 * s12 = lo12 + (i + u(w1)) cw12 and s13 = lo13 + (j + u(w2)) cw13 in float32
 * (u(w) = (w >> 40) 2^-24, cw = (float)(box width / cells)); accepted when the point is in
 * the kinematic region and u(w3) * bound[c] < |S|^2 (float32). */
typedef struct goo_envelope {
  int32_t n12, n13;
  const float* bound;       /* n12 * n13 values                                            */
} goo_envelope;
typedef struct goo_server_options {
  int64_t hbm_budget_bytes; /* event arena (<= 0: half of the free device memory)           */
  int32_t max_fits;         /* fit slots (<= 0: 4096)                                       */
  int32_t tile_events;      /* events per tile of the batched launch (<= 0: 16384)          */
  int32_t max_iter;         /* BFGS iterations per fit (<= 0: 200)                          */
  int32_t pad;
  double edm_tol;           /* (<= 0: 1e-6)                                                 */
  const goo_envelope* envelope; /* NULL: 1.2 x the 3x3-neighbourhood maximum of |S|^2 over a
                               96 x 96 grid, 6 x 6 lattice points per cell                 */
} goo_server_options;
int goo_server_create(goo_model* model, const double* theta_gen, const int* free_mask, const double* scale,
                      const goo_server_options* options, goo_server** out);
int goo_server_submit(goo_server* server, int64_t n_events, uint64_t seed, const double* theta_start,
                      int64_t* ticket);
int goo_server_step(goo_server* server, int* n_queued, int* n_active, int* n_done);
int goo_server_result(goo_server* server, int64_t ticket, double* theta_out, double* errors_out,
                      goo_fit_result* res);
/* The tickets of fits that finished (converged, failed, cancelled or refused admission) since
 * the previous call, oldest first: up to `cap` of them are written to tickets[0..*n) and
 * removed from the list; the rest wait for the next call (*n == cap: call again).  A study
 * of many toy fits (Sec. 5, toy MC studies) collects results this way instead
 * of asking for every outstanding ticket after each step.  The results stay available to
 * goo_server_result.  GOO_ERR_ARG for a NULL server or n, cap < 0, or cap > 0 with NULL
 * tickets. */
int goo_server_finished(goo_server* server, int64_t* tickets, int cap, int* n);
/* Failures of one served fit leave the others untouched (each fit's evaluation depends only on
 * its own tiles and theta).  goo_server_submit refuses a non-finite theta_start with
 * GOO_ERR_ARG; nothing is queued.  goo_server_cancel ends a queued or active fit between
 * steps: a queued one leaves the queue, an active one releases its slot and its events'
 * memory; its result is theta_start with zero errors, nll = +inf and status
 * GOO_FIT_CANCELLED.  GOO_ERR_STATE for a finished fit, GOO_ERR_ARG for an unknown ticket.
 * goo_server_fail_allocation is a failure-detection test hook: the admission of that queued
 * fit fails as if its event memory could not be allocated, and the fit ends with status
 * GOO_FIT_ALLOC_FAILED while the queue moves on (GOO_ERR_STATE unless the fit is queued). */
enum { GOO_FIT_ALLOC_FAILED = 6, GOO_FIT_CANCELLED = 7 };
int goo_server_cancel(goo_server* server, int64_t ticket);
int goo_server_fail_allocation(goo_server* server, int64_t ticket);
/* out[0..8]: evaluation rounds, evaluation ms, generation ms, candidates drawn, candidates
   accepted, largest envelope bound, arena bytes, arena bytes in use, and the candidates inside
   the region whose |S|^2 exceeded their cell's bound (non-zero: the envelope is too low there
   and the toys under-populate those points). */
int goo_server_stats(const goo_server* server, double* out /* 9 doubles */);
int goo_server_free(goo_server* server);
/* Toys from the same generator, written to host float arrays: one toy, or n_toys toys
 * generated together (toy i at offset n[0] + ... + n[i-1]); a toy does not depend on the
 * others it is generated with. */
int goo_toy_generate(goo_model* model, const double* theta, const goo_envelope* env, uint64_t seed,
                     int64_t n_events, float* s12_out, float* s13_out);
int goo_toys_generate(goo_model* model, const double* theta, const goo_envelope* env, int n_toys, const uint64_t* seeds,
                      const int64_t* n_events, float* s12_out, float* s13_out);
/* NLL and gradient of n_fits (dataset, theta) pairs of one amplitude model in one launch
 * (FP32 path); theta: n_fits x n_params, nll_out: n_fits, grad_out: n_fits x n_params.  The
 * fits must share every non-coefficient parameter. */
int goo_nll_grad_batch(goo_model* model, int n_fits, const goo_dataset* const* datasets, const double* theta,
                       int precision, double* nll_out, double* grad_out);

/* ---- shards (paper Sec. 4: MPI divides the dataset among processes) --------------------------
 * Partial sums over events [begin, end) of ds: out[0] = sum of -log f, out[1] = its
 * compensation term, out[2] = number of events, out[3 .. 3+n_params) = gradient partials
 * (zero unless want_grad).  The normalisation is computed in full by every shard.
 * goo_combine_partials adds n_parts such records (stride 3+n_params) in index order with
 * compensated arithmetic into out (same layout); nll = out[0] + out[1]. */
int goo_nll_partial(goo_model* model, const goo_dataset* ds, int64_t begin, int64_t end,
                    const double* theta, int precision, int want_grad, double* out);
/* End-to-end evaluation from host memory with the transfer overlapped (paper Sec. 1: the time
 * of a fit is the per-event evaluation; Fig. 1: a DataSet feeds the PDF).  Refills ds (an
 * owning dataset of capacity >= n_events, as goo_dataset_update would) from n_events events
 * of pinned float32 host columns (host_cols[c], one per dataset column) and returns the FP32
 * NLL and adjoint gradient of a sum-of-products model at theta over them.  The events are
 * split into n_chunks (1..64) chunks on multiples of 3072 events (the event kernel's column
 * tile): the copy engine moves chunk
 * c + 1 over the host link (on a second stream of the context) while chunk c is converted to
 * float64, range-checked and evaluated on the context's stream, so that only the last
 * chunk's evaluation follows the transfer.  The chunks' records are added in chunk order with
 * compensation.  GOO_ERR_RANGE (*n_bad = count, ds left empty) if any event lies outside its
 * observable's limits; GOO_ERR_UNSUPPORTED for amplitude models; other errors as goo_nll_grad.
 * The call returns when the result is on the host. */
int goo_nll_grad_streamed(goo_model* model, goo_dataset* ds, const float* const* host_cols, int64_t n_events,
                          int n_chunks, const double* theta, double* nll_out, double* grad_out, int64_t* n_bad);
int goo_combine_partials(int n_parts, int n_params, const double* parts, double* out);

/* ---- Faddeeva function ------------------------------------------------------------------
 * w(z) = exp(-z^2) erfc(-i z) for Im z >= 0 by the library's rational approximation
 * (Weideman 1994; 24 terms for GOO_F32, evaluated in float, 40 terms for GOO_F64), the
 * function the four-body model's decay-time resolution uses.  Host-only: it lets the
 * arithmetic the kernels run be checked on the CPU.  out[0] = Re w, out[1] = Im w. */
int goo_faddeeva(double re, double im, int precision, double* out);

/* ---- FMA-pipe peaks -------------------------------------------------------------------------
 * The paper quotes advertised single- and double-precision FLOP/s of its GPUs (Table 1); this
 * call measures them on the context's device, as the denominators of the FP64 and FP32
 * rooflines.  One launch of num_sms x 4 blocks of 256 threads, each thread running 8
 * independent chains of iters x 16 fused multiply-adds, timed with CUDA events on ctx's stream
 * after one untimed launch.  kind: GOO_PEAK_F64 (fma.rn.f64), GOO_PEAK_F32 (fma.rn.f32) or
 * GOO_PEAK_F32X2 (packed fma.rn.f32x2, two FMAs per instruction).  fma_per_s (host) receives
 * FMAs per second (FLOP/s = 2 x that), ms_out (host, nullable) the launch's duration.
 * GOO_ERR_ARG for a NULL pointer, an unknown kind or iters outside 1 .. 2^24. */
enum { GOO_PEAK_F64 = 0, GOO_PEAK_F32 = 1, GOO_PEAK_F32X2 = 2 };
int goo_peak_fma(goo_ctx* ctx, int kind, int iters, double* fma_per_s, double* ms_out);

/* ---- likelihood without device allocation ------------------------------------------------
 * The paper has no counterpart to this call.  It computes the same NLL and gradient as
 * goo_nll_grad for a sum/product model, but allocates nothing: no goo_ctx, goo_dataset or
 * goo_model is needed.  It serves callers that cannot call cudaMalloc -- code running where
 * another component owns all device memory (an application's own pool, a host framework
 * whose allocator forbids side allocations) or code that cannot pay the implicit device
 * synchronisation and latency of cudaMalloc/cudaFree on every call.
 *
 *   nodes..obs_hi, norm  the model exactly as for goo_model_build / goo_model_set_norm, but
 *                        limited to two levels: a leaf, a PROD of leaves, or an ADD of leaves
 *                        and PRODs of leaves; GOO_NORM_ANALYTIC or GOO_NORM_GRID.
 *   cols_dev             n_obs device column pointers (16-byte aligned) of n_events values:
 *                        float for GOO_F32, double for GOO_F64.  Not range-checked.
 *   theta, nll_out, grad_out   host arrays as for goo_nll_grad.
 *   cuda_stream          stream for the work (NULL: the legacy default stream).
 *
 * All intermediate device state lives in one file-scope device array of 1 MiB, which every
 * GPU that loads the library holds until the process exits.  Maximum sizes: n_params <= 32,
 * n_obs <= 4, <= 4 products of <= 4 leaves; larger requests fail with GOO_ERR_ARG or
 * GOO_ERR_UNSUPPORTED and a message.  Every call looks up the array's device address
 * (cudaGetSymbolAddress, which allocates nothing) with the caller's current device, so the
 * call keeps working after a cudaDeviceReset.  Every call reuses the same array and clears
 * its counters first; the array keeps the previous call's contents otherwise.  Calls that
 * overlap on the GPU (different streams or host threads, same device) race on the array:
 * serialise them.  The call copies the model block in and the result out on cuda_stream and
 * synchronises that stream before it returns, so it cannot be captured in a CUDA graph (both
 * the copies from pageable host memory and the synchronisation are refused during a stream
 * capture).  GOO_ERR_NONPOSITIVE_PDF and GOO_ERR_TIMEOUT as for goo_nll_grad (nll_out = +inf,
 * grad_out zeroed). */
int goo_nll_grad_static(const goo_node* nodes, int n_nodes, int n_params, int n_obs, const double* obs_lo,
                        const double* obs_hi, const goo_norm_spec* norm, const void* const* cols_dev,
                        int precision, int64_t n_events, const double* theta, void* cuda_stream,
                        double* nll_out, double* grad_out);

#ifdef __cplusplus
}
#endif

#endif /* GOO_H */
