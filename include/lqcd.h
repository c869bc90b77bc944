/*
 * lqcd.h -- C ABI of liblqcd, a GB300 (sm_103a) library for site-wise lattice
 * field expressions and stout link smearing on a periodic 4D lattice.
 *
 * Sources of the operations (cited per entry point below):
 *   [W]   F. Winter, "Accelerating QDP++ using GPUs" (arXiv:1105.2279):
 *         Sec. 4.2 (flattened expression evaluation, shift site tables),
 *         Sec. 4.4 (thread geometry N_threads / N_site, auto-tuning),
 *         Sec. 5 (device residency API), Sec. 6 Listing 1 (shift, adj,
 *         products, the Jacobi smearing routine), Sec. 8 (coalesced layout,
 *         auto-tuning as next steps).
 *   [MP]  C. Morningstar, M. Peardon, Phys. Rev. D 69 (2004) 054501:
 *         Sec. II (stout link), Sec. III (Cayley-Hamilton exp(iQ)),
 *         Sec. IV (stout force recursion).
 *
 * Conventions shared by every call
 *   - Lattice dims (Lx, Ly, Lz, Lt); mu = 0,1,2,3 = x,y,z,t; site index
 *     s = x + Lx*(y + Ly*(z + Lz*t)); periodic in every direction.
 *     A link U_mu(x) sits on the bond x -> x + mu.
 *   - Device layout (structure of arrays, component-major): an element is a
 *     complex number stored as (re, im) = float2 / double2, except kind
 *     LQ_REAL (one float / double).  A field of kind k holds
 *     [ndir][ncomp][V] elements with (ndir, ncomp) = LINKS (4, 9),
 *     COLOR_MATRIX (1, 9), COLOR_VECTOR (1, 3), COMPLEX (1, 1), REAL (1, 1),
 *     FERMION (1, 12); matrix component c = 3*row + col, fermion component
 *     c = 3*spin + colour.  Consecutive threads read
 *     consecutive sites of one component plane (coalesced 8/16 B vectors).
 *   - Host interchange layout (AoS, the QDP++ site-major order):
 *     [V][ndir][ncomp] elements of the field's precision, (re, im)
 *     interleaved.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on it, except those that return host values
 *     (reductions, plaquette, upload/download), which synchronise it.
 *   - Every call returns an lq_status; on error nothing is launched, output
 *     fields are left untouched and lq_last_error() describes the failure.
 *     No call aborts, traps or prints.
 *   - Ownership: handles (lq_geom, lq_field) belong to the caller and are
 *     released with the matching destroy/free call; memory passed to
 *     lq_field_wrap stays owned by the caller; host buffers are never kept.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int lq_status;
#define LQ_OK                0
#define LQ_ERR_ARG          (-1)  /* invalid argument (NULL, range, aliasing)           */
#define LQ_ERR_GEOM         (-2)  /* fields on different geometries / wrong kind        */
#define LQ_ERR_OOM          (-3)  /* device allocation failed                           */
#define LQ_ERR_CUDA         (-4)  /* a CUDA runtime call failed                         */
#define LQ_ERR_TIMEOUT      (-5)  /* a bounded device-side wait gave up                 */
#define LQ_ERR_NUMERIC      (-6)  /* non-finite value detected where checked            */
#define LQ_ERR_UNSUPPORTED  (-7)  /* valid request this build does not implement        */

typedef enum lq_kind {
  LQ_LINKS = 0, LQ_COLOR_MATRIX = 1, LQ_COLOR_VECTOR = 2, LQ_COMPLEX = 3, LQ_REAL = 4, LQ_FERMION = 5
} lq_kind;

typedef enum lq_prec { LQ_F32 = 0, LQ_F64 = 1 } lq_prec;

typedef struct lq_geom lq_geom;    /* opaque: lattice dims and volume        */
typedef struct lq_field lq_field;  /* opaque: geometry, kind, prec, device ptr */

/* Thread-local description of the last error of this thread ("" if none). */
const char* lq_last_error(void);

/* ABI version of this header (1). */
int lq_abi_version(void);

/* ---- geometry and fields ([W] Sec. 5; layout [W] Sec. 8) -------------- */

/* dims: 4 ints >= 1 with Lx*Ly*Lz*Lt < 2^31.  *out receives a new handle. */
lq_status lq_geom_create(const int dims[4], lq_geom** out);
lq_status lq_geom_destroy(lq_geom* g);
/* Volume V and dims of a geometry. */
lq_status lq_geom_info(const lq_geom* g, int dims_out[4], long long* volume_out);

/* Bytes of a field of (kind, prec) on g: V * ndir * ncomp * element size. */
lq_status lq_field_bytes(const lq_geom* g, int kind, int prec, size_t* bytes_out);

/* Allocates a device field owned by the library (stream-ordered on `stream`,
 * contents undefined); release with lq_field_free.  Counterpart of the
 * paper's pushToLattice() allocation ([W] Sec. 5). */
lq_status lq_field_alloc(const lq_geom* g, int kind, int prec, void* stream, lq_field** out);

/* Wraps caller-owned device memory (e.g. a torch tensor) as a field.
 * dev_ptr must be 16-byte aligned and hold at least lq_field_bytes(). */
lq_status lq_field_wrap(const lq_geom* g, int kind, int prec, void* dev_ptr, size_t bytes,
                        lq_field** out);

/* Releases the handle; frees the memory only if the library allocated it
 * (freeDeviceMem(), [W] Sec. 5). */
lq_status lq_field_free(lq_field* f);

/* Device pointer of a field (structure-of-arrays layout above). */
lq_status lq_field_device_ptr(const lq_field* f, void** ptr_out);

/* Host AoS -> device SoA ([W] Sec. 5 pushToLattice copy).  host_aos holds
 * lq_field_bytes() bytes in the host interchange layout; it is read before
 * the call returns (the stream is synchronised).  Page-locked host memory
 * (cudaHostAlloc / cudaHostRegister, which the GPU addresses directly) is
 * read by the transpose kernel itself over the host link; pageable memory
 * is copied into a device staging buffer first. */
lq_status lq_field_upload(lq_field* f, const void* host_aos, void* stream);

/* Device SoA -> host AoS ([W] Sec. 5 popFromLattice copy); page-locked host
 * memory is written by the transpose kernel directly, pageable memory through
 * a staging buffer and a copy.  Synchronises. */
lq_status lq_field_download(const lq_field* f, void* host_aos, void* stream);

/* Field checkpoints on disk (checkpoint / resume of smeared fields).  File:
 * a 48-byte little-endian header -- magic "LQFIELD1", int32 version (1),
 * int32 kind, int32 prec, int32 dims[4], int32 0, int64 payload bytes --
 * followed by the field in the host interchange (AoS) layout.  Save
 * downloads and writes; load checks the header against the field (dims, kind,
 * precision: LQ_ERR_GEOM on mismatch, LQ_ERR_ARG for a file that is not a
 * field checkpoint) before uploading.  Both synchronise `stream`; the host
 * staging buffer is allocated and freed inside the call. */
lq_status lq_field_save(const lq_field* f, const char* path, void* stream);
lq_status lq_field_load(lq_field* f, const char* path, void* stream);

/* ---- site-wise operations ([W] Sec. 6 Listing 1) ------------------------ */

/* out(x) = in(x + sign*mu), periodic: sign = +1 is QDP++ FORWARD, -1
 * BACKWARD (Listing 1).  out and in: same geometry, kind and precision,
 * distinct memory.  No site table is read: neighbours are index arithmetic. */
lq_status lq_shift(lq_field* out, const lq_field* in, int mu, int sign, void* stream);

/* Flattened expression program ([W] Sec. 4.2): a per-site register machine
 * over 3x3 complex matrices.  A COLOR_VECTOR operand is loaded into column 0
 * (other columns zero) and stored from column 0; COMPLEX/REAL operands load
 * as scalar * identity and store the (0,0) entry. */
enum {
  LQ_OP_LOAD = 0,   /* r[dst] = shift(operand[a] (dir `dir` if LINKS), sign, mu); sign 0: no shift */
  LQ_OP_ADJ = 1,    /* r[dst] = r[a]^dagger                                       */
  LQ_OP_MUL = 2,    /* r[dst] = r[a] * r[b]                                       */
  LQ_OP_ADD = 3,    /* r[dst] = r[a] + r[b]                                       */
  LQ_OP_SUB = 4,    /* r[dst] = r[a] - r[b]                                       */
  LQ_OP_SCALE = 5,  /* r[dst] = (re + i im) * r[a]                                */
  LQ_OP_TRACE = 6,  /* r[dst] = tr(r[a]) * 1                                      */
  LQ_OP_RETR = 7,   /* r[dst] = Re tr(r[a]) * 1                                   */
  LQ_OP_STORE = 8   /* result = r[a]                                              */
};
#define LQ_EXPR_MAX_OPS 64
#define LQ_EXPR_MAX_REGS 8
#define LQ_EXPR_MAX_OPERANDS 8
typedef struct lq_op {
  int code, dst, a, b;   /* opcode and register / operand indices            */
  int dir, mu, sign;     /* LOAD: link direction, shift direction and sign   */
  int pad;
  double re, im;         /* SCALE factor                                      */
} lq_op;

/* Evaluates `prog` at every site.  operands: n_operands fields of one
 * geometry and precision.  If out_or_null is given (kind COLOR_MATRIX,
 * COLOR_VECTOR, COMPLEX or REAL), the stored register is written to it.  If
 * reduce_out_or_null is given, it receives sum_x tr(result(x)) as
 * (re, im), accumulated in FP64 in a fixed order (run-to-run bit identical);
 * the stream is then synchronised.  The program must end with one STORE. */
lq_status lq_expr_eval(lq_field* out_or_null, const lq_op* prog, int n_ops,
                       const lq_field* const* operands, int n_operands,
                       double* reduce_out_or_null, void* stream);

/* JIT-compiled form of lq_expr_eval ([W] Sec. 4.1: one kernel compiled per
 * expression at run time and kept loaded; Sec. 8: compiled once across
 * runs).  The program becomes straight-line CUDA C (registers as locals,
 * kinds and shifts as constants) compiled by NVRTC for sm_103a; the cubin is
 * cached in memory per program text and device, and on disk when
 * lq_jit_cache_dir() names a directory.  Same arguments, validation and
 * results (bit for bit) as lq_expr_eval.  Returns LQ_ERR_UNSUPPORTED if
 * libnvrtc cannot be loaded; compilation errors come back as LQ_ERR_CUDA with
 * the NVRTC log in lq_last_error(). */
lq_status lq_expr_eval_jit(lq_field* out_or_null, const lq_op* prog, int n_ops,
                           const lq_field* const* operands, int n_operands,
                           double* reduce_out_or_null, void* stream);

/* Compiles (or finds in the caches) the kernel lq_expr_eval_jit would run for
 * this program, fields and reduction flag, without launching anything: the
 * "compile before production" step.  Needs no GPU. */
lq_status lq_expr_jit_prepare(const lq_field* out_or_null, const lq_op* prog, int n_ops,
                              const lq_field* const* operands, int n_operands, int reduce);

/* Directory for compiled expression kernels kept across runs (NULL or ""
 * disables the disk cache).  Files: lqjit_<hash>.cu (the source, compared on
 * lookup) and lqjit_<hash>.cubin. */
lq_status lq_jit_cache_dir(const char* path);

/* out[0..3] = NVRTC compilations, in-memory cache hits, disk cache hits,
 * module loads, since the library was loaded. */
lq_status lq_jit_stats(long long out[4]);

/* ---- global reductions (FP64 accumulation, deterministic) ---------------- */

/* out[0..1] = sum over sites and components (re, im); REAL fields give im = 0. */
lq_status lq_reduce_sum(const lq_field* f, double out[2], void* stream);

/* out[0..1] = sum_x tr M(x) for COLOR_MATRIX; sum_x sum_mu tr U_mu(x) for LINKS. */
lq_status lq_reduce_trace(const lq_field* f, double out[2], void* stream);

/* Average plaquette of a LINKS field:
 *   out[0] = (1/(18V)) sum_x sum_{mu<nu} Re tr P_{mu nu}(x)   (unit field -> 1),
 *   out[1] = spatial planes (nu < 3), out[2] = temporal planes, each / (9V),
 * with P_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag.
 * Products in the field precision, accumulation in FP64.  Synchronises. */
lq_status lq_plaquette(const lq_field* links, double out[3], void* stream);

/* Unnormalised plaquette sums over the sites [s_begin, s_end) only:
 * out[0] = sum of Re tr P over the 3 spatial planes, out[1] = over the 3
 * temporal planes, products and accumulation as in lq_plaquette (fixed
 * reduction tree for a given range size).  A rank of a domain-decomposed
 * lattice sums its interior sites and the ranks add their sums (one FP64
 * all-reduce of two numbers).  0 <= s_begin <= s_end <= volume.
 * Synchronises. */
lq_status lq_plaquette_sums(const lq_field* links, long long s_begin, long long s_end, double out[2],
                            void* stream);

/* Wilson action S = beta sum_x sum_{mu<nu} (1 - Re tr P_{mu nu}(x)/3). */
lq_status lq_wilson_action(const lq_field* links, double beta, double* out, void* stream);

/* ---- stout smearing ([MP] Secs. II-IV) ------------------------------------ */

typedef struct lq_stout_opts {
  int struct_size;        /* sizeof(lq_stout_opts); 0 => all defaults               */
  int reproject;          /* -1 default (on for LQ_F32 links, off for LQ_F64), 0, 1 */
  int use_graph;          /* 1: record the n-step launch sequence as a CUDA graph
                             and replay it.  The recorded graph and its links-sized
                             workspace are kept per (field pointer, dims, n, rho,
                             dirs, launch shape, device) until lq_free_all; at most
                             8 are kept (least recently launched dropped first).
                             Calls with the same key share that workspace, so two
                             such calls must not overlap on the GPU.                */
  int variant;            /* 0 tuned/default, 1 global-load kernel,
                             2 shared-memory staged kernel (FP32 links),
                             3 two kernels per step: the two-link products
                               U_mu(y) U_nu(y+mu) of every ordered pair of smeared
                               directions, then the staples from them (9 products
                               per link instead of 12; a scratch buffer of
                               |dirs|(|dirs|-1) colour-matrix fields).  Variants 0-2
                               give bit-identical links; variant 3 associates the
                               staple products differently (equal to rounding), so
                               the tuner never picks it: it is requested here.      */
  int block;              /* threads per block (N_threads, [W] Sec. 4.4); 0 = tuned  */
  int sites_per_thread;   /* N_site ([W] Sec. 4.4); 0 = tuned                        */
  void* work;             /* optional device workspace of >= one links field;
                             NULL => the library allocates it stream-ordered         */
  size_t work_bytes;
} lq_stout_opts;

/* n_steps stout steps in place on a LINKS field.  dirs_mask bit mu selects
 * smeared directions; staples sum over nu in dirs, nu != mu; links outside
 * dirs are unchanged.  Each step computes every new link from the previous
 * step's field (double-buffered internally).  Precision follows the field:
 *   LQ_F64: all arithmetic FP64.
 *   LQ_F32: staples, Omega, Q, exp assembly and U' = exp(iQ) U in FP32;
 *           Cayley-Hamilton coefficients f0,f1,f2 in FP64; SU(3)
 *           re-projection of every new link (unless reproject = 0): the
 *           Gram-Schmidt of rows 0 and 1 with row 2 = conj(row0 x row1),
 *           its cancelling sums (row norms - 1, row overlap, row0 x row1)
 *           in FP64 and its small corrections applied in FP32; the result
 *           is the FP64 Gram-Schmidt rounded to FP32, except for elements
 *           within ~1e-12 of an FP32 rounding boundary, which may differ by
 *           one unit in the last place.
 *           Stated accuracy (max per-element |U - U_exact|, up to 6 steps,
 *           measured on GB300): 3e-7 on near-identity fields (plaquette
 *           ~0.6), 4e-7 over a whole 48^3 x 96 lattice, 6e-7 on Haar-random
 *           fields with rho <= 0.4; it does not grow with the step count.
 * The coefficients come from [MP] Sec. III's closed form, or, for
 * c1 = tr(Q^2)/2 <= 3/4, from the Taylor series of exp(iQ) reduced with
 * Q^3 = c1 Q + c0, truncated where its error bound is under 1e-17 (FP64
 * links) or 1e-10 (FP32 links, whose coefficients are rounded to FP32).
 * rho >= 0 and finite; n_steps >= 0; dirs_mask in [1, 15]. */
lq_status lq_stout_smear(lq_field* links_inout, double rho, int n_steps, unsigned dirs_mask,
                         const lq_stout_opts* opts, void* stream);

/* Stout smearing of links in HOST memory, end to end, with the transfers
 * overlapped with the arithmetic.  host_in / host_out: the AoS link layout
 * of lq_field_upload / lq_field_download for `geom` and `prec` (host_out
 * may equal host_in; page-locked memory lets the copies run asynchronously).
 * The lattice is cut into n_chunks slabs of whole t-slices (0: 16, at most
 * dims[3]); each slab is copied and transposed to the device layout as it
 * arrives, the first step of a slab starts once it and its two neighbouring
 * slabs are resident, and each slab of the final field is transposed back
 * and copied out as soon as its last step is done.  Arithmetic, rules and
 * results are those of lq_stout_smear (bit for bit, global-load kernel; the
 * launch shape comes from opts->block, else a cached tuning result, else the
 * default).  plaq_out (optional, 3 doubles) receives lq_plaquette of the
 * result.  Device memory: three link fields from the library pool.
 * Synchronizes the stream.  ([W] Sec. 4.3 moves fields between host and
 * device on demand; here the transfers run behind the smearing.) */
lq_status lq_stout_smear_host(const void* host_in, void* host_out, const lq_geom* geom, int prec, double rho,
                              int n_steps, unsigned dirs_mask, int n_chunks, double* plaq_out,
                              const lq_stout_opts* opts, void* stream);

/* One stout step from `in` into `out` over the sites [s_begin, s_end) only
 * (site index x + Lx (y + Ly (z + Lz t))): for those sites and the
 * directions in dirs_mask, out receives exactly the links lq_stout_smear's
 * step would produce (same kernel and arithmetic, global-load variant; the
 * launch shape from opts->block / sites_per_thread, else a cached tuning
 * result, else the default); every other site and direction of out is left
 * as it was.  This is the step of a domain-decomposed smearing ([W] Sec. 8
 * names multi-GPU parallelisation as future work): a rank holding a slab of
 * t-slices plus one halo slice on each side smears the slab's interior
 * slices, whose staples read at most one slice away.  in and out: LINKS of
 * one geometry and precision, distinct memory; 0 <= s_begin <= s_end <=
 * volume; rho finite >= 0; dirs_mask in [1, 15].  Asynchronous. */
lq_status lq_stout_step_range(const lq_field* in, lq_field* out, double rho, unsigned dirs_mask,
                              long long s_begin, long long s_end, const lq_stout_opts* opts, void* stream);

/* Coefficient-stage statistics of n_steps stout steps of `links` (which is
 * not modified; the steps run on library scratch copies with the default
 * launch shape and precision rules of lq_stout_smear).  counts[0] = link
 * updates, counts[1] = updates whose Cayley-Hamilton coefficients took the
 * truncated Taylor series (c1 <= 3/4), counts[2] = the sum of their series
 * orders K (degree 2K+1).  The paper has no counterpart: this is
 * instrumentation for counting the FP64 work of the coefficient stage, whose
 * size depends on the field.  Synchronizes the stream. */
lq_status lq_stout_ch_stats(const lq_field* links, double rho, int n_steps, unsigned dirs_mask,
                            long long* counts, void* stream);

typedef struct lq_backward_opts {
  int struct_size;        /* sizeof(lq_backward_opts); 0 => defaults                */
  int checkpoint_every;   /* k >= 1: keep U^(j) for j % k == 0 and recompute the
                             others forward from the nearest kept field; 1 (default)
                             keeps every step                                        */
} lq_backward_opts;

/* Gradient of a scalar S(stout^n(U)) with respect to the thin links U.
 *   grad_seed: LINKS field G_n = dS/dRe U^(n) + i dS/dIm U^(n); NULL =>
 *              S is the Wilson action of the smeared field at `beta`.
 *   force_out: LINKS field receiving F_mu(x) = TA(G_mu(x) U_mu(x)^dag)
 *              (traceless anti-Hermitian; d/de S(exp(eX)U_mu(x)) = Re tr F^dag X).
 *   grad_out:  optional LINKS field receiving G w.r.t. the thin links.
 * The recursion is the stout force of [MP] Sec. IV, evaluated with the same
 * precision rules as lq_stout_smear (FP32 links: FP32 matrix algebra, FP64
 * coefficients).  One kernel per step runs the staple gather of step j+1
 * and the link stage of step j on each link.  Scratch memory is allocated
 * stream-ordered: the kept checkpoints, two gradient fields, two fields of
 * the staple-sum gradient, one link field for U^(n) (Wilson seed only) and,
 * when checkpoint_every > 1, three link fields for the recomputation. */
lq_status lq_stout_backward(const lq_field* thin_links, double rho, int n_steps, unsigned dirs_mask,
                            const lq_field* grad_seed, double beta, lq_field* force_out,
                            lq_field* grad_out, const lq_backward_opts* opts, void* stream);

/* One step of the stout force recursion of lq_stout_backward ([MP]
 * Sec. IV), on the sites [s_begin, s_end) of LINKS fields of one geometry
 * and precision: for callers that hold one part of a lattice (a t-slab with
 * a halo slice on each side, see lq_stout_step_range; [W] Sec. 8 names
 * multi-GPU parallelisation as future work) and run the recursion step by
 * step, exchanging halos in between.  With U^(j+1) = stout step of U^(j):
 *   G' = the gradient at U^(j+1) of the link, from `source`:
 *     LQ_BWD_SOURCE_WILSON: -(beta/3) (sum of the staples of u_next, all
 *                           planes): the Wilson action of U^(j+1) = u_next;
 *     LQ_BWD_SOURCE_GIVEN:  g_in (a seed dS/dU^(j+1));
 *     LQ_BWD_SOURCE_GATHER: g_in (G_U(local) of step j+1) plus the six
 *                           staple-insertion terms of k_next (K of step j+1)
 *                           on u_next (= U^(j+1)), for smeared directions;
 *   with k_out (a link stage, u_cur = U^(j)): g_out = G_U(local) and
 *     k_out = K (the gradient w.r.t. the bare staple sum) of step j, for the
 *     directions in dirs_mask; other directions get g_out = G' and k_out
 *     untouched;
 *   without k_out (the last step, u_cur = the thin links): g_out (optional)
 *     = G', the gradient at the thin links, and force_out (optional) =
 *     TA(G' u_cur^dag).
 * Reads of u_next, k_next and u_cur reach at most one site away from the
 * range in every direction; g_in and the outputs only the range itself.
 * Sites outside the range are left as they were.  Outputs must not alias
 * each other or an input.  rho finite >= 0, beta finite, 0 <= s_begin <=
 * s_end <= volume.  Results equal those of lq_stout_backward (checkpoints
 * kept every step) bit for bit.  Asynchronous. */
#define LQ_BWD_SOURCE_WILSON 0
#define LQ_BWD_SOURCE_GIVEN 1
#define LQ_BWD_SOURCE_GATHER 2
lq_status lq_stout_backward_step(const lq_field* u_next, const lq_field* k_next, const lq_field* g_in,
                                 const lq_field* u_cur, lq_field* g_out, lq_field* k_out, lq_field* force_out,
                                 int source, double rho, double beta, unsigned dirs_mask, long long s_begin,
                                 long long s_end, void* stream);

/* Smears n_cfg independent LINKS fields (any geometries, one precision) with
 * one persistent launch per step over a device work list of (config, tile)
 * items; with opts->use_graph the n-step sequence is a replayed CUDA graph.
 * Results equal n_cfg separate lq_stout_smear calls bit for bit.
 * Memory: the work list (n_cfg descriptors) is kept per (field pointers,
 * dims, launch shape, dirs, device), at most 16 lists, least recently used
 * dropped first.  Without use_graph the double buffer (the size of all the
 * fields together) and the step counters come stream-ordered from the
 * library pool on every call and go back to it at the end of the call.  With
 * use_graph the recorded graph owns its double buffer and counters, kept per
 * (work-list key, n_steps, rho, reproject) until lq_free_all, at most 4
 * graphs; calls with the same graph key share them, so two such calls must
 * not overlap on the GPU. */
lq_status lq_stout_smear_batch(lq_field* const* links, int n_cfg, double rho, int n_steps,
                               unsigned dirs_mask, const lq_stout_opts* opts, void* stream);

/* APE smearing (Albanese et al., Phys. Lett. B 192 (1987) 163; the paper
 * has no counterpart: an adjacent smearing on the stout step's staple sum),
 * n_steps steps in place on a LINKS field:
 *   V_mu(x) = (1 - alpha) U_mu(x) + alpha / (2 (d - 1)) * C_mu(x),  d = |dirs|,
 *   U'_mu(x) = W exp(-i arg(det W) / 3),  W = V (V^dag V)^(-1/2)  (polar factor),
 * C_mu the staple sum of lq_stout_smear (without rho), arg in (-pi, pi].
 * The mixing runs in the field precision, the projection in FP64.  V must
 * be non-singular (a singular V gives NaN).  alpha finite; n_steps >= 0;
 * dirs_mask in [1, 15]; links outside dirs are unchanged. */
lq_status lq_ape_smear(lq_field* links_inout, double alpha, int n_steps, unsigned dirs_mask, void* stream);

/* Gradient of a scalar S(ape^n(U)) with respect to the thin links U: the
 * fat-link force of APE smearing (the paper has no counterpart).  Arguments,
 * outputs, checkpoints, scratch and errors as in lq_stout_backward, with
 * alpha and dirs_mask as in lq_ape_smear (grad_seed NULL => the Wilson
 * action of the smeared field at `beta`).  Per step and smeared link, the
 * gradient G' at U' = P(V) goes to G_V through the projection:
 *   U' = W z, z = (det W)^(-1/3):  G_W = conj(z) G' + (i/3) Im tr(G'^dag U') W
 *   W = V (V^dag V)^(-1/2):       G_V = (G_W - 2 W Y) Z^-1,  Z = (V^dag V)^(1/2),
 *                                 Y the solution of Z Y + Y Z = Herm(V^dag G_W)
 * and from G_V to the links: (1 - alpha) G_V on U_mu(x) itself and
 * alpha / (2 (d - 1)) G_V through each staple, as in the stout force.
 * FP32 links: staples, mixing and staple gradients in FP32, the projection
 * and its gradient in FP64.  V must be non-singular. */
lq_status lq_ape_backward(const lq_field* thin_links, double alpha, int n_steps, unsigned dirs_mask,
                          const lq_field* grad_seed, double beta, lq_field* force_out,
                          lq_field* grad_out, const lq_backward_opts* opts, void* stream);

/* HYP smearing (Hasenfratz and Knechtli, Phys. Rev. D 64 (2001) 034504; the
 * paper has no counterpart), n_steps steps in place on a LINKS field, all
 * four directions: three nested APE-type levels with weights a3 (innermost,
 * 2 staples), a2 (4 staples) and a1 (outermost, 6 staples), whose staples
 * stay inside the hypercubes attached to the link, each level projected to
 * SU(3) as in lq_ape_smear; usual weights (a1, a2, a3) = (0.75, 0.6, 0.3).
 * Staples and mixing in the field precision, projections in FP64.  Scratch:
 * 24 colour-matrix fields of decorated links and one link field. */
lq_status lq_hyp_smear(lq_field* links_inout, double a1, double a2, double a3, int n_steps, void* stream);

/* Gradient of a scalar S(hyp^n(U)) with respect to the thin links U: the
 * fat-link force of HYP smearing (the paper has no counterpart).  Arguments,
 * outputs, checkpoints and errors as in lq_stout_backward, with the weights
 * of lq_hyp_smear (all four directions smeared).  Per step the three levels
 * run backwards: the gradient at each level's sum V goes through the
 * projection's gradient of lq_ape_backward, then into the decorated links
 * (or thin links) that the level's staples read, through the staple
 * gradient with K = (level weight / staple count) G_V; each link also
 * collects (1 - a_i) G_V of the sums it enters directly.  Staples, mixing
 * and staple gradients in the field precision, projections and their
 * gradients in FP64.  Scratch: 64 colour-matrix fields (decorated links and
 * their gradients) besides the checkpoints. */
lq_status lq_hyp_backward(const lq_field* thin_links, double a1, double a2, double a3, int n_steps,
                          const lq_field* grad_seed, double beta, lq_field* force_out,
                          lq_field* grad_out, const lq_backward_opts* opts, void* stream);

/* ---- Jacobi smearing ([W] Sec. 6, Listing 1 and the operator K) ----------- */

/* n_iter Jacobi smearing iterations of a quark field, in place:
 *   s0 = chi;  repeat n_iter times:
 *     chi(x) <- s0(x) + kappa * sum_{mu in dirs} [U_mu(x) chi(x+mu) + U_mu(x-mu)^dag chi(x-mu)]
 *   then chi /= norm
 * (Listing 1; the hopping term is the off-diagonal part of the operator K).
 * links: LINKS field; chi: COLOR_VECTOR (3 complex per site) or FERMION
 * (4 spins x 3 colours; the links act on colour, every spin alike); same
 * geometry and precision.  dirs_mask selects the summed directions (Listing 1
 * sums all four; 7 leaves out t, like a smearing that skips the time
 * direction).  norm != 0.  One fused kernel per iteration (hopping term, axpy
 * and, in the last iteration, the 1/norm scaling) over two ping-pong buffers;
 * scratch: s0 and one work copy of chi, allocated stream-ordered. */
lq_status lq_jacobi_smear(const lq_field* links, lq_field* chi_inout, double kappa, int n_iter, double norm,
                          unsigned dirs_mask, void* stream);

typedef struct lq_jacobi_opts {
  int struct_size;        /* sizeof(lq_jacobi_opts); 0 => defaults                  */
  int compress_links;     /* 1: the iterations read rows 0 and 1 of each link from a
                             packed copy (made once per call, 2/3 of the link
                             bytes) and rebuild row 2 = conj(row0 x row1); exact for
                             SU(3) links, to rounding for links unitary to
                             rounding; wrong for links outside SU(3).  0: off    */
  int block;              /* N_threads ([W] Sec. 4.4): threads per block, a multiple
                             of 32 in [32, 256]; 0 = tuned (lq_tune on) or 128   */
  int sites_per_thread;   /* N_site ([W] Sec. 4.4): sites per thread in [1, 64];
                             0 = tuned (lq_tune on) or 1.  With the tuner on and
                             neither field set, the first call per (field kind,
                             link storage, precision, dims, dirs, device) times
                             N_threads in {32,64,128,256} x N_site in {1,2,4,8}
                             on two iterations in its work buffers and keeps the
                             fastest.  Any shape gives bit-identical results.   */
} lq_jacobi_opts;

/* lq_jacobi_smear with options (opts NULL => lq_jacobi_smear).  Compressed
 * links cut the HBM traffic of each iteration; the paper has no counterpart
 * (its Sec. 8 names the memory layout as the next optimisation). */
lq_status lq_jacobi_smear_ex(const lq_field* links, lq_field* chi_inout, double kappa, int n_iter, double norm,
                             unsigned dirs_mask, const lq_jacobi_opts* opts, void* stream);

/* exp(iQ) of every matrix of a COLOR_MATRIX field of Hermitian traceless Q,
 * through the same Cayley-Hamilton evaluation as the stout step ([MP]
 * Sec. III): coefficients f0, f1, f2 in FP64 from c0 = det Q and
 * c1 = tr(Q^2)/2, then f0 + f1 Q + f2 Q^2 in the field precision.  Only the
 * Hermitian part of each input is read (upper triangle and real diagonal;
 * the trace is removed in FP64).  out and q: same geometry and precision,
 * distinct memory. */
lq_status lq_expiq(lq_field* out, const lq_field* q, void* stream);

/* Stout smearing that allocates no device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot let a library
 * allocate -- applications whose own allocator already holds all device
 * memory, plug-ins whose host forbids device allocations, and latency-critical
 * paths that must not risk an allocation's synchronisation or failure.
 * Same arguments and results as lq_stout_smear with default options (FP32
 * links re-projected, no graph), but the double buffer is a built-in device
 * array of LQ_NOALLOC_WORK_BYTES (32 MiB) that every GPU loading the library
 * holds until the process exits; fields needing more return LQ_ERR_ARG
 * (FP64 up to 58,254 sites, FP32 up to 116,508 sites).  The first call on each
 * device looks the array's device address up (cudaGetSymbolAddress); make that
 * first call before any stream capture.  All calls share the one array, so
 * calls whose work overlaps on the GPU (different streams, or different host
 * threads on one device) race; serialise them.  The array keeps the last
 * call's contents; nothing in it needs to start at zero. */
#define LQ_NOALLOC_WORK_BYTES (32u * 1024u * 1024u)
lq_status lq_stout_smear_noalloc(lq_field* links_inout, double rho, int n_steps, unsigned dirs_mask, void* stream);

/* ---- auto-tuning ([W] Sec. 4.4 and Sec. 8) and device storage ------------- */

/* Enables the auto-tuner: the first smearing call per (kernel, precision,
 * dims, device) times the candidate block sizes and N_site values on a
 * scratch copy and keeps the fastest.  cache_path (may be NULL) names a
 * text file that is read now and rewritten after each new entry. */
lq_status lq_tune(const char* cache_path);

/* The tuned (block, sites_per_thread, variant) for a key, if known. */
lq_status lq_tune_lookup(int prec, const int dims[4], unsigned dirs_mask, int* block,
                         int* sites_per_thread, int* variant);

/* ---- measurement ---------------------------------------------------------- */

/* CUDA-core FMA throughput of the current device, measured: a grid of 8 CTAs
 * of 256 threads per SM, each thread running eight independent FMA chains in
 * precision prec (LQ_F32 or LQ_F64), one untimed launch and one timed with
 * CUDA events on `stream` (~20 ms).  *tflops receives 2 x FMAs / time in
 * TFLOP/s: the measured peak of the FP32 and FP64 pipes, the denominators of
 * the rooflines of kernels bound by them.  The paper has no counterpart.
 * Synchronizes the stream. */
lq_status lq_peak_probe(int prec, double* tflops, void* stream);

/* Releases every cache the library holds on the device (workspaces, graphs,
 * descriptor tables), like theDeviceStorage::freeAll() ([W] Sec. 5).
 * Fields are not touched. */
lq_status lq_free_all(void);

#ifdef __cplusplus
}
#endif
#endif /* LQCD_H */
