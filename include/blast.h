/*
 * blast.h — C ABI of the GB300 beyond-Limber angular power spectrum library.
 *
 * The library computes, for every pair of tomographic tracers, the angular
 * power spectrum of Eq. cls-general of Chiarenza et al. (arXiv:2410.03632),
 *
 *   C^{AB}_ij(l) = N_AB(l) int dchi1 W^A_i(chi1) int dchi2 W^B_j(chi2)
 *                  int dk k^2 P(k, chi1, chi2) j_l(k chi1) j_l(k chi2) / ((k chi1)^a (k chi2)^b),
 *
 * without the Limber approximation, by the paper's method (Sec. 3):
 *   (pre) basis integrals T~^{AB}_{n;l}(chi1, chi2) of Eq. t_tilde, once per grid;
 *   (a0)  Chebyshev coefficients of P (Eqs. chebpoints, a2, dft, cheb_pk);
 *   (a)   projected matter density w_l = sum_n c_n T~_{n;l} (Eq. pmd);
 *   (b)   the chi-R quadrature of Eq. final_cls in its unsymmetrised form
 *         (Eq. app1 with chi2 = R chi1) and the probe prefactor N_AB(l) of
 *         Eqs. gg, ss, gs.
 * The power spectrum is growth separable, P(k, chi1, chi2) = D(chi1) D(chi2) P(k)
 * (Sec. 4.2.1), so c_n(chi1, chi2) = D(chi1) D(chi2) a_n.
 *
 * Units: chi in Mpc/h, k in h/Mpc.  Tracer types: g = clustering, s = lensing.
 * Spectrum (pair) order in every output: gg (i <= j, row major), then gs
 * (i clustering, j lensing, all pairs, row major), then ss (i <= j).
 * Output arrays are row major C[pair][ell], ells in plan order restricted to
 * the request's ell mask.
 *
 * Conventions for every entry point:
 *   - the return value is a blast_status (0 = success, negative = error);
 *   - on BLAST_EINVAL nothing is written to any output;
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream);
 *   - the library owns plans, basis tables, work space and servers; the caller
 *     owns request arrays and output arrays;
 *   - a plan may be used by one call at a time (its work space is reused);
 *     concurrent evaluation goes through a server, which owns per-slot space;
 *   - pointers tagged "host or device" follow the request's mem_space.
 */
#ifndef BLAST_H
#define BLAST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct blast_plan blast_plan;
typedef struct blast_server blast_server;
typedef struct blast_graph blast_graph;

typedef enum {
    BLAST_OK = 0,
    BLAST_EINVAL = -1,    /* bad argument; no output written */
    BLAST_ENOMEM = -2,    /* device or host allocation failed, or over budget */
    BLAST_ENOTREADY = -3, /* result not ready yet (poll) */
    BLAST_ETIMEOUT = -4,  /* a bounded wait ran out */
    BLAST_EDEVICE = -5,   /* a CUDA call failed */
    BLAST_ENOBASIS = -6,  /* the requested precision's basis table is absent */
    BLAST_EBUSY = -7      /* server queue full */
} blast_status;

/* Arithmetic of contraction (a) and quadrature (b).  The Chebyshev fit and the
 * basis precompute are always FP64. */
typedef enum {
    BLAST_FP64 = 0,   /* FP64 on CUDA cores (reference GPU path) */
    BLAST_FP32 = 1,   /* FP32 basis, FP32 CUDA-core contraction, FP64 final sums */
    BLAST_BF16S = 2   /* batched tcgen05 contraction on BF16 tensor cores: the
                         coefficients and each basis column are cut into five
                         8-bit fixed-point slices held exactly in BF16; the 15
                         slice products of total order <= 4 accumulate exactly
                         in five FP32 TMEM levels, which a cascade of exact
                         two-sums combines, so the Chebyshev sum keeps about 40
                         bits through the strong cancellation of Eq. pmd where
                         P(k) is small; the R sum runs on compensated FP32 pairs
                         (e_ij about 2e-5 against FP64 on the 3x2pt grid) */
} blast_precision;

/* Bits of the precisions_mask of blast_precompute_basis. */
#define BLAST_BASIS_FP64 (1u << 0)
#define BLAST_BASIS_FP32 (1u << 1)
#define BLAST_BASIS_BF16S (1u << 2)  /* slice tables of the tensor-core path */

/* Grid and size description of a plan (Sec. 3.2 of the paper).
 *   ell      n_ell integer multipoles, 2 <= ell, strictly increasing, n_ell <= 128;
 *            ignored when ell_real is set
 *   ell_real NULL, or n_ell real multipoles, 2 <= ell <= 1e5, strictly increasing
 *            (App. A evaluates the basis at l = 211.63): the basis uses spherical
 *            Bessel functions of that real order, N_AB(l) and the Limber terms
 *            take l as given.  Integer values give the integer plan exactly.
 *   chi      n_chi evenly spaced nodes on [chi_min, chi_max], composite Simpson
 *            weights (3/8 rule on the last three intervals when n_chi is even)
 *   R        r_form 0 (the split form, chi2 = R chi1 with R in [R_min, R_max]):
 *            n_R nodes, two panels [R_min, 1] and [1, R_max] of n_R/2 first-kind
 *            Chebyshev points each with Fejer-1 weights (n_R even, R_min < 1 < R_max);
 *            r_form 1 (the symmetrised form of App. A, Eq. app1: R in (0, 1] and
 *            C_ij = N_AB sum wchi wR chi [K^A_i(chi) K^B_j(R chi) + K^B_j(chi) K^A_i(R chi)] w):
 *            the n_R positive points of the (2 n_R + 1)-point first-kind Chebyshev
 *            rule on [-1, 1] with its Fejer-1 weights (the even extension of the R
 *            integrand; the middle node R = 0 carries j_l(0) = 0); R_min and R_max
 *            are ignored.  Plans of r_form 1 serve every precision;
 *            blast_cl_nonsep refuses them (BLAST_EINVAL)
 *   k        n_cheb Chebyshev coefficients over [k_min, k_max]; k_map 0 maps k
 *            linearly onto [-1, 1], k_map 1 maps ln k linearly
 *   n_kquad  Clenshaw-Curtis points of the basis k integral, 2^m + 1
 *   max_clust, max_lens  largest tracer counts a request may carry
 *   device   CUDA device ordinal that holds the plan's tables
 *   r_form   0 or 1, see R                                                   */
typedef struct {
    int n_ell;
    const int32_t *ell;
    int n_chi;
    double chi_min, chi_max;
    int n_R;
    double R_min, R_max;
    int n_cheb;
    double k_min, k_max;
    int k_map;
    int n_kquad;
    int max_clust, max_lens;
    int device;
    int r_form;
    const double *ell_real;
} blast_plan_desc;

/* One cosmology.  Tracers 0..n_clust-1 are clustering, n_clust..n_clust+n_lens-1
 * lensing; kernels are the paper's calligraphic K of Eq. final_cls (lensing
 * kernels already divided by chi^2).  All arrays float64, row major, host or
 * device per mem_space.  When they are read: a call with host outputs waits for
 * its stream, so every input is read before it returns; a call with device
 * outputs is stream ordered, so device inputs, and pinned host inputs (copied
 * with cudaMemcpyAsync), are read when the stream runs the call (pageable host
 * inputs are staged before it returns) and must stay unchanged until then.
 *   kern_chi     [n_clust+n_lens][n_chi]          K at chi_a
 *   kern_Rchi    [n_clust+n_lens][n_chi*n_R]      K at R_r chi_a, index a*n_R + r
 *   growth_chi   [n_chi]                          D(chi_a)
 *   growth_Rchi  [n_chi*n_R]                      D(R_r chi_a)
 *   k_tab, p_tab [n_ptab] linear P(k): k strictly increasing, P > 0, 3 <= n_ptab <= 1024,
 *                and [k_tab[0], k_tab[n_ptab-1]] must contain every Chebyshev k-node
 *   ell_mask_lo/hi  bit e selects plan ell e (lo: e < 64, hi: 64 <= e < 128); 0,0 = all
 *   mem_space    0 = host pointers, 1 = device pointers                      */
typedef struct {
    int n_clust, n_lens;
    const double *kern_chi;
    const double *kern_Rchi;
    const double *growth_chi;
    const double *growth_Rchi;
    int n_ptab;
    const double *k_tab;
    const double *p_tab;
    uint64_t ell_mask_lo, ell_mask_hi;
    int mem_space;
} blast_request;

/* Build a plan: host grids (Simpson, Fejer-1, Clenshaw-Curtis weights, Chebyshev
 * nodes) and device tables for desc->device.  The basis is NOT computed here.
 * Errors: BLAST_EINVAL (bad description), BLAST_ENOMEM, BLAST_EDEVICE.      */
int blast_plan_create(const blast_plan_desc *desc, blast_plan **out);

/* Free a plan and every device buffer it owns.  NULL is accepted. */
int blast_plan_destroy(blast_plan *plan);

/* Copy the plan's nodes to host arrays (any of them may be NULL):
 * chi[n_chi], R[n_R], k_cheb[n_cheb] (the k of each Chebyshev point t_j =
 * cos((2j+1) pi / 2 n_cheb), Eq. chebpoints).  Callers sample their kernels
 * and growth at chi_a and R_r chi_a. */
int blast_plan_nodes(const blast_plan *plan, double *chi, double *R, double *k_cheb);

/* Number of spectra for a tracer count, in the pair order above. */
int blast_npairs(int n_clust, int n_lens);

/* Step (pre), Eq. t_tilde: compute T~^{AB}_{n;l}(chi_a, R_r chi_a) for the
 * three types gg (f = k^2), gs (f = 1), ss (f = 1/k^2) in FP64 on the device,
 * then derive the copies named in precisions_mask (FP64 is always kept).
 * Synchronous with respect to the host when it returns.  Errors: BLAST_EDEVICE. */
int blast_precompute_basis(blast_plan *plan, unsigned precisions_mask, void *stream);

/* Copy the FP64 basis between the plan and a caller buffer of
 * 3*n_ell*n_cheb*n_chi*n_R doubles laid out [type][ell][n][a*n_R + r]
 * (mem_space 0 host, 1 device).  basis_set replaces the basis and rebuilds the
 * reduced-precision copies named in precisions_mask.  Errors: BLAST_ENOBASIS
 * (get before any basis exists), BLAST_EDEVICE. */
int blast_basis_get(const blast_plan *plan, double *dst, int mem_space, void *stream);
int blast_basis_set(blast_plan *plan, const double *src, int mem_space,
                    unsigned precisions_mask, void *stream);

/* Save / load the FP64 basis to a file with a header (magic, grid sizes, grid
 * checksum) and a payload checksum; load rejects a file made for another grid
 * with BLAST_EINVAL and rebuilds the reduced-precision copies in precisions_mask. */
int blast_basis_save(const blast_plan *plan, const char *path);
int blast_basis_load(blast_plan *plan, const char *path, unsigned precisions_mask);

/* Steps (a0), (a), (b) for one cosmology.  cl_out[npairs][n_sel] receives FP64
 * C_l (n_sel = ells selected by the mask), host or device per out_mem_space.
 * With a host output the call waits for the stream; otherwise it is stream
 * ordered.  BLAST_BF16S runs the same tensor-core kernel as a batch of one.
 * Errors: BLAST_EINVAL, BLAST_ENOBASIS, BLAST_EDEVICE, BLAST_ETIMEOUT (a bounded
 * device wait of an earlier or this call gave up; the call's outputs are void). */
int blast_cl(blast_plan *plan, const blast_request *req, int precision,
             double *cl_out, int out_mem_space, void *stream);

/* The same for n cosmologies in one pass: every request has its own P(k),
 * kernels, growth, tracer counts (<= the plan maxima) and ell mask.  outs[i]
 * receives request i's C (layout as blast_cl).  BLAST_BF16S runs contraction
 * (a) as one tcgen05 GEMM over the batch (cosmologies x Chebyshev order x
 * chi-R nodes) with the R sum of quadrature (b) fused in its epilogue; it
 * needs n_R a multiple of 32, n_cheb <= 96 and at most 10 tracers of each
 * kind (BLAST_EINVAL otherwise). */
int blast_cl_batch(blast_plan *plan, int n, const blast_request *reqs, int precision,
                   double *const *outs, int out_mem_space, void *stream);

/* Non-separable spectrum (Eqs. cheb_pk and pmd with a general c_n(chi1, chi2):
 * scale-dependent growth, massive neutrinos).  p_nodes[q][j] = P(k_j, chi_a,
 * R_r chi_a) at the Chebyshev k-nodes k_j of blast_plan_nodes for every chi-R
 * node q = a n_R + r, [n_chi n_R][n_cheb] doubles in the request's memory
 * space.  Per node the coefficients are fitted in FP64 on the device (the
 * transform of the separable fit), w_l = sum_n c_n(q) T~_{n;l}(q), and the
 * chi-R quadrature is the FP64 one.  The request's growth arrays still
 * multiply the kernels (pass ones when p_nodes carries the whole time
 * dependence); its P table is checked as for blast_cl but not used.
 * cl_out as blast_cl.  Errors as blast_cl. */
int blast_cl_nonsep(blast_plan *plan, const blast_request *req, const double *p_nodes, double *cl_out,
                    int out_mem_space, void *stream);

/* ---------------------------------------------------------------- Limber
 * The Limber approximation of Sec. 2.2 on the plan's chi rule,
 *   C^Limber_ij(l) = pref_AB(l) sum_a wchi_a / chi_a^2 W_i(chi_a) W_j(chi_a) P(nu / chi_a, chi_a),
 * nu = l + 1/2, pref = 1 (gg), sqrt((l+2)(l+1)l(l-1)) / nu^2 (gs),
 * (l+2)(l+1)l(l-1) / nu^4 (ss), W = the clustering kernel, or the lensing
 * kernel times chi^2 (requests carry lensing kernels divided by chi^2).
 *
 * blast_limber_k: the Limber points k[e][a] = (ell_e + 1/2) / chi_a,
 *   [n_ell][n_chi] host doubles, at which a caller samples its non-linear P.
 * blast_cl_limber: C^Limber for one request (no basis needed), cl_out as
 *   blast_cl.  p_nl NULL: the request's linear spectrum, D(chi_a)^2 P(k) with
 *   P(k) from its table by the natural cubic spline in (ln k, ln P) of the
 *   Chebyshev fit, zero outside the table; extended = 1 adds the first-order
 *   (extended Limber) correction: each term times
 *   1 - [chi^2/2 (Kt_i''/Kt_i + Kt_j''/Kt_j) + chi^3/6 (Kt_i'''/Kt_i + Kt_j'''/Kt_j)] / nu^2,
 *   Kt = W D / sqrt(chi), derivatives by central differences on the chi nodes
 *   (needs n_chi >= 5).  p_nl set: P[e][a] at the Limber points for every
 *   plan ell, [n_ell][n_chi] doubles in the request's memory space, used as
 *   given (growth included by the caller); extended must then be 0.
 * blast_cl_nonlinear: the total spectrum of Sec. 3.2,
 *   C_tot = C_lin + C^Limber(P_delta) - C^Limber(P_lin),
 *   C_lin the beyond-Limber C_l at `precision`, p_nl = P_delta at the Limber
 *   points as above; the correction vanishes when p_nl holds the linear P.
 * Errors as blast_cl (BLAST_EINVAL also for a misaligned p_nl). */
int blast_limber_k(const blast_plan *plan, double *k);
int blast_cl_limber(blast_plan *plan, const blast_request *req, const double *p_nl, int extended, double *cl_out,
                    int out_mem_space, void *stream);
int blast_cl_nonlinear(blast_plan *plan, const blast_request *req, int precision, const double *p_nl,
                       double *cl_out, int out_mem_space, void *stream);

/* Coefficient envelope of BLAST_BF16S.  The five slices hold each cosmology's
 * Chebyshev coefficients to 40 bits of its largest one; since the coefficients
 * of a power spectrum fall by decades with n, basis row n is scaled by a power
 * of two s_n and the coefficients by 1 / s_n (exact, the products unchanged),
 * so every term a_n T~_n keeps its 40 bits.  env[n_cheb] > 0 gives the shape
 * (rounded to powers of two, at most 2^16 below its maximum); NULL restores
 * the default, the running maximum of the coefficients of a generic linear
 * power spectrum x / (1 + x^3), x = k / 0.02 h/Mpc, held at or above 2^-8 of
 * its first value (tabulated spectra keep high-n coefficients of that
 * order; an envelope below a cosmology's own coefficients costs precision
 * instead of gaining it).  The slice tables are
 * rebuilt if present.  Errors: BLAST_EINVAL (a non-positive entry),
 * BLAST_EDEVICE. */
int blast_set_coef_envelope(blast_plan *plan, const double *env);

/* Allocation-free evaluation.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory while evaluating,
 * for example a host framework that has reserved the GPU's memory for its own
 * pool allocator (a cudaMalloc behind its back can fail or fragment the pool)
 * or a latency-critical request loop (cudaMalloc / cudaFree can synchronise
 * the device and stall other streams).
 * It computes the same FP64 C_l as blast_cl(plan, req, BLAST_FP64, ...) but
 * takes all scratch (coefficients, weights, partial sums, descriptors) from a
 * fixed device array of BLAST_NOALLOC_SCRATCH_BYTES compiled into the library,
 * which every GPU that loads the library holds until the process exits.  It
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *   req       device inputs only (req->mem_space must be 1), else BLAST_EINVAL;
 *             checked as blast_cl checks them (tracer counts, table size, ell
 *             mask bits inside the plan), and every pointer, cl_out included,
 *             must be 8-byte aligned (BLAST_EINVAL otherwise, nothing launched)
 *   cl_out    device array [npairs][n_sel], written on the stream
 *   returns   BLAST_ENOMEM when the request needs more scratch than the array
 *             holds (about 3 n_ell n_chi max_tracers + (n_clust+n_lens)
 *             n_chi n_R doubles; the 3x2pt 10+10-bin 100-ell grid fits),
 *             BLAST_ENOBASIS without an FP64 basis, BLAST_EDEVICE on CUDA errors.
 * Set-up happens in blast_plan_create, on the plan's device with that device
 * current: it looks up the array's device address and loads the code of the
 * kernels this path launches (CUDA loads modules lazily), so the array's
 * memory is taken when the plan is made and the call itself takes none.  All
 * calls share the one array, whose contents persist between calls: every byte
 * a call reads is written earlier in the same call, and calls that overlap on
 * the GPU (other streams, other host threads) race on it. */
#define BLAST_NOALLOC_SCRATCH_BYTES (16u << 20)
int blast_cl_noalloc(blast_plan *plan, const blast_request *req, double *cl_out, void *stream);

/* Device bytes one request occupies while in flight in blast_cl (inputs,
 * coefficients, weights, partial sums, outputs): a sizing aid for callers. */
size_t blast_request_footprint(const blast_plan *plan, const blast_request *req);

/* ---------------------------------------------------------------- serving
 * A server evaluates requests submitted from any host thread by continuous
 * batching over one or more resident plans (Sec. 3.3: the basis is computed
 * once and reused for every cosmology; requests share it).
 *
 * blast_server_create: plans[0..n_plans) stay owned by the caller, must outlive
 *   the server, and must not be used by other calls while it exists (its
 *   workers use their work space); a plan may appear once.  Each plan gets a
 *   lane: a worker thread, a stream, the plan's work space reserved for
 *   batches of max_slots requests, and a ring of 2 max_slots device slots, each
 *   holding the inputs and the C_l of the largest request the plan accepts (one
 *   batch running while the next forms).  All of it is allocated here; no
 *   device memory is allocated afterwards.  hbm_budget bounds the device bytes
 *   reserved in total (blast_server_reserved): BLAST_ENOMEM if they exceed it
 *   or an allocation fails, BLAST_EINVAL for a repeated or null plan.
 * blast_server_reserved: device bytes the server holds (0 for null).
 * blast_submit: copies the request's inputs (host or device, per mem_space)
 *   into server-owned pinned memory before it returns, checks them as
 *   blast_cl would (BLAST_EINVAL, BLAST_ENOBASIS; n_ptab at most 1024), and
 *   admits the request when its plan's ring has a free slot and the queue
 *   (16 max_slots) has room, else BLAST_EBUSY (retry later; a slot frees when
 *   its batch ends).  *ticket identifies it.  A lane's oldest waiting request
 *   fixes the precision of the lane's next batch; its waiting requests with
 *   that precision join in arrival order, up to max_slots.  Lanes run
 *   concurrently.  A request's C_l does not depend on its batch or on the
 *   other lanes (FP64 bitwise equal to blast_cl; BF16S bitwise equal to the
 *   request evaluated alone).  A batch that fails is re-run request by
 *   request, so a bad request fails alone.
 * blast_poll: waits up to timeout_us microseconds (negative = until done) for
 *   the ticket.  Not done: BLAST_ENOTREADY, *done = 0.  Done: *done = 1, the
 *   request's status is returned, on success C[npairs][n_sel] is copied to
 *   cl_out (host or device memory), and the ticket is retired (polling it
 *   again is BLAST_EINVAL, as is an unknown ticket).
 * blast_server_destroy: evaluates the requests still waiting, frees results
 *   never polled, and frees the server; no call on the server may run
 *   concurrently with it. */
int blast_server_create(blast_plan *const *plans, int n_plans, size_t hbm_budget, int max_slots,
                        blast_server **out);
int blast_submit(blast_server *server, int plan_idx, const blast_request *req, int precision, uint64_t *ticket);
int blast_poll(blast_server *server, uint64_t ticket, double *cl_out, int *done, int64_t timeout_us);
int blast_server_destroy(blast_server *server);
size_t blast_server_reserved(const blast_server *server);

/* ---------------------------------------------------------------- batch graphs
 * One blast_cl_batch call captured into a CUDA graph for repeated launches with
 * the same buffers (Sec. 3.3: the basis is computed once and every cosmology
 * reuses it; a sampler evaluates new parameters in the same arrays).
 * blast_graph_create: reqs[0..n) with device inputs (mem_space 1) and outs[i]
 *   device arrays [npairs][n_sel] (8-byte aligned), checked as blast_cl_batch
 *   checks them (BLAST_EINVAL, BLAST_ENOBASIS; BLAST_ETIMEOUT as blast_cl).  It
 *   stages the request descriptors, allocates a work space the graph owns
 *   (blast_graph_reserved bytes) and captures the call's kernels; synchronous.
 *   The pointers, tracer counts, P-table lengths and ell masks of reqs are
 *   fixed in the graph; the contents of every input array may change between
 *   launches.  The plan must outlive the graph, and its basis must not be
 *   replaced or reloaded while the graph exists.
 * blast_graph_launch: enqueues the kernels on stream (stream ordered; the
 *   outputs are complete when the stream reaches the end of the launch).
 *   BLAST_ETIMEOUT when a bounded device wait of an earlier launch or call on
 *   the plan gave up.  Launches and other calls on the same plan must not
 *   overlap on the GPU.
 * blast_graph_destroy: frees the graph and its work space (NULL: EINVAL). */
int blast_graph_create(blast_plan *plan, int n, const blast_request *reqs, int precision, double *const *outs,
                       blast_graph **out);
int blast_graph_launch(blast_graph *graph, void *stream);
size_t blast_graph_reserved(const blast_graph *graph);
int blast_graph_destroy(blast_graph *graph);

/* Kernel classes of the evaluation path, for blast_profile_read. */
#define BLAST_K_FIT 0         /* step (a0): Chebyshev fit */
#define BLAST_K_WEIGHTS 1     /* quadrature weights U, V with growth folded in */
#define BLAST_K_CONTRACT 2    /* steps (a) + (b, sum over R) on CUDA cores */
#define BLAST_K_CONTRACT_TC 3 /* steps (a) + (b, sum over R) on tcgen05 tensor cores */
#define BLAST_K_REDUCE 4      /* step (b, sum over chi) and prefactor */
#define BLAST_K_CLASSES 5

/* Per-kernel device time.  While enabled, every evaluation call brackets each
 * of its kernel launches with CUDA events recorded on the stream the kernel
 * runs on (the call's stream, or the plan's side stream of the fit).
 * blast_profile_read waits for those events and returns, for one kernel class,
 * the summed device milliseconds and the launch count since the last reset
 * (launches are counted whether or not timing is enabled). */
int blast_profile_enable(blast_plan *plan, int enable);
int blast_profile_read(blast_plan *plan, int kernel_class, double *total_ms, long long *launches);
int blast_profile_reset(blast_plan *plan);

/* Test hook of the bounded device waits.  The next BLAST_BF16S call on the
 * plan has one epilogue warp of its first CTA wait, before tile `tile`, on a
 * barrier that nothing completes, with a limit of 2e7 clock cycles; the wait
 * runs out, the kernel records the error word and every warp leaves after its
 * copies and MMAs in flight complete, and the call returns BLAST_ETIMEOUT (a
 * host-output call at once, a device-output call on the next call).  The
 * context stays usable; -1 cancels.  Errors: BLAST_EINVAL. */
int blast_test_trip_wait(blast_plan *plan, int tile);

/* Autotuner of the BLAST_BF16S launch parameters: the contraction's number
 * of persistent CTAs and the reduction's chi-chunk warps and stages per warp.
 * The candidates run the caller's representative batch reqs[0..n) (device
 * outputs the call allocates and frees) under the kernel timer; the fastest
 * set stays in the plan for later calls of any batch size.  cache_path
 * (optional) is a text file keyed by GPU name, plan dimensions and cosmology
 * tiles: a key found there is used without timing; a new choice is appended.
 * The tuned set never changes a result beyond the summation order of the
 * chi sum.  Errors: BLAST_EINVAL (plan not served by the tensor cores),
 * BLAST_ENOBASIS, BLAST_ENOMEM, and those of blast_cl_batch.
 * blast_tuned_params reads the current set (0 = built-in choice). */
int blast_autotune(blast_plan *plan, int n, const blast_request *reqs, const char *cache_path, void *stream);
int blast_tuned_params(const blast_plan *plan, int *grid, int *red_warps, int *red_stages);

/* Human-readable name of a status code (static string). */
const char *blast_status_str(int status);

#ifdef __cplusplus
}
#endif
#endif /* BLAST_H */
