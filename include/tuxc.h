/*
 * tuxc.h -- C ABI of the GB300 Tucker-tensor Fock-exchange library (libtuxc.so).
 *
 * The library applies the Fock exchange operator of a block of real orbitals on a
 * tensor-product grid, following arXiv 2401.04189 ("Convolution operation" section):
 *
 *   (K psi)_i(r) = - sum_j psi_j(r) * phi_ij(r),     phi_ij = conv(psi_i psi_j, 1/|r|)
 *                                                    (Eqs. ExchangeOperator, varphi, hadam)
 *
 * with every pair density projected onto a shared Tucker basis U1, U2, U3 (Eq. tucker,
 * Eq. TuckerDecompField) and 1/r replaced by a sum of T Gaussians (Eq. gauss), so that the
 * 3-D convolution is a weighted sum of tensor products of 1-D convolutions (Eq. final),
 * each evaluated with nodal quadrature as a matrix product (Eq. discInteg):
 *
 *   rho_ij = psi_i * psi_j
 *   G_ij   = rho_ij x1 U1^T x2 U2^T x3 U3^T                               [r1][r2][r3]
 *   A_td   = C_td U_d,  C_td[a][b] = w_b exp(-theta_t (x_a - x_b)^2)       [n_d][r_d]
 *   phi_ij = sum_t mu_t G_ij x1 A_t1 x2 A_t2 x3 A_t3                       [n1][n2][n3]
 *   W_i    = - sum_j psi_j * phi_ij
 *   E_x    = 1/2 sum_i sum_r w(r) psi_i(r) W_i(r)       (exact-exchange energy, alpha = 1)
 *
 * Occupations are 1, there is no spin factor and alpha = 1: callers scale.
 *
 * Conventions for every entry point
 *  - Orbital blocks are float32, C-contiguous [count][n1][n2][n3] (z fastest), in device
 *    memory of the current CUDA device, 16-byte aligned.  Outputs must not overlap inputs
 *    (an overlap is rejected with TX_ERR_INVALID_ARG).
 *  - Every call is asynchronous on the caller's stream; nothing is synchronised.  Scalars
 *    (energies) are written to caller-owned device memory.
 *  - Every call returns a status: TX_OK (0) or a negative TX_ERR_* code.  Arguments are
 *    validated on the host before any launch; a failed validation launches nothing.
 *    No exception or abort crosses the ABI.  tx_status_string() names a code;
 *    tx_last_error_message() gives the detail of the last failure on this thread.
 *  - A context belongs to one device and must be used from one host thread at a time.
 */
#ifndef TUXC_H
#define TUXC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* tx_stream_t;   /* same object as cudaStream_t; NULL = legacy default stream */
typedef struct tx_ctx tx_ctx;

enum tx_status {
    TX_OK = 0,
    TX_ERR_INVALID_ARG = -1,          /* null pointer, non-positive size, non-finite value */
    TX_ERR_SHAPE = -2,                /* rank larger than grid size, inconsistent extents */
    TX_ERR_NOT_ORTHONORMAL = -3,      /* U_d^T U_d deviates from I by more than 1e-10 */
    TX_ERR_UNSUPPORTED_PRECISION = -4,
    TX_ERR_CUDA = -5,                 /* a CUDA runtime call failed; see tx_last_error_message */
    TX_ERR_OOM = -6,                  /* device allocation for the context workspace failed */
    TX_ERR_TIMEOUT = -7,              /* a bounded device-side wait gave up (see tx_check_device_error) */
    TX_ERR_NOT_SETUP = -8,            /* NULL or destroyed context */
    TX_ERR_UNSUPPORTED_SHAPE = -9,    /* shape outside what the selected precision's kernels handle */
    TX_ERR_ALIGNMENT = -10,           /* a device pointer is not 16-byte aligned */
    TX_ERR_NOT_DEFINITE = -11         /* ACE: the exchange matrix is not negative definite */
};

/* Arithmetic of the mode-product GEMMs.  Accumulation is float32 in every mode; set-up
 * (the A_td matrices) and the final energy reduction are float64. */
enum tx_precision {
    TX_PREC_FP32 = 0,     /* plain float32 CUDA-core kernels (reference GPU form) */
    TX_PREC_BF16 = 1,     /* tcgen05 kind::f16, bf16 operands, fp32 accumulate in TMEM */
    TX_PREC_TF32 = 2,     /* tcgen05 kind::tf32, one pass */
    TX_PREC_TF32X3 = 3,   /* tcgen05 kind::tf32, split precision: hi*hi + hi*lo + lo*hi */
    TX_PREC_BF16X3 = 4    /* tcgen05 kind::f16, bf16 split precision: hi*hi + hi*lo + lo*hi */
};

/*
 * tx_tucker_setup -- build a context for one grid, basis and Gaussian sum.
 *
 * Defines the operator of Eqs. tucker, gauss, quadVal and discInteg (the 1-D convolution
 * matrices are precomputed once, as the paper does after Eq. discInteg).
 *   n[3]              grid sizes n1, n2, n3 (>= 2)
 *   x1, x2, x3        host float64 node coordinates, n_d each
 *   w1, w2, w3        host float64 quadrature weights, n_d each (> 0)
 *   r[3]              Tucker ranks (1 <= r_d <= n_d)
 *   U1, U2, U3        host float64 [n_d][r_d] row-major, U_d^T U_d = I (checked to 1e-10)
 *   T                 number of Gaussian terms (>= 1)
 *   gauss_exponents   host float64 theta[T] (> 0)
 *   gauss_weights     host float64 mu[T] (finite, > 0)
 *   precision         enum tx_precision
 *   stream            stream for the set-up copies and kernels
 * The host arrays are copied; the caller may free them when the call returns.  A_td is
 * computed on the device in float64 (mu_t folded into A_t3 before rounding) and rounded
 * to the operand formats of `precision`.  On success *ctx owns all its device memory and
 * is released by tx_destroy.  On failure *ctx is set to NULL.
 */
int tx_tucker_setup(tx_ctx** ctx, const int n[3],
                    const double* x1, const double* x2, const double* x3,
                    const double* w1, const double* w2, const double* w3,
                    const int r[3], const double* U1, const double* U2, const double* U3,
                    int T, const double* gauss_exponents, const double* gauss_weights,
                    int precision, tx_stream_t stream);

/*
 * tx_exchange_apply_galerkin / tx_exchange_energy_galerkin -- the same calls with the convolution
 * projected onto the Tucker basis on both sides.  The one-sided operator of Eq. final is C P,
 * P = (x)_d U_d U_d^T; this form applies P^* C P, where P^* = D^-1 P D is the adjoint of P in the
 * inner product weighted by the quadrature weights D:
 *     phi_ij = (sum_t mu_t G_ij x_d B_td) x_d (D_d^-1 U_d),     B_td = U_d^T D_d A_td  (r_d x r_d)
 *     W_i    = - sum_j psi_j * phi_ij
 *     E_x    = - 1/2 sum_ij <G_ij, sum_t mu_t G_ij x_d B_td>     (in core space, O(T r^4) per pair)
 * With the nodal quadrature the exchange matrix <psi_a, W_b>_w is then exactly symmetric and
 * negative semi-definite at any rank (the one-sided form is so only at full rank).  Arguments,
 * layouts, aliasing rules and errors are those of tx_exchange_apply / tx_exchange_energy.  Both
 * run in float32 on the CUDA cores whatever the context's precision.
 */
int tx_exchange_apply_galerkin(tx_ctx* ctx, const float* psi_occ, int n_occ, const float* psi_tgt, int n_tgt,
                               float* out, tx_stream_t stream);
int tx_exchange_energy_galerkin(tx_ctx* ctx, const float* psi_occ, int n_occ, double* e_dev, tx_stream_t stream);

/*
 * tx_exchange_apply_sthosvd -- out = K psi_tgt with per-pair Tucker bases, the paper's own
 * decomposition (Eq. TuckerDecompField): every pair density rho_ij = psi_i psi_j gets its bases
 * from a sequentially truncated HOSVD (modes 1, 2, 3 in turn: U_d,ij = the r_d leading
 * eigenvectors of the Gram matrix of the mode-d unfolding of the partly projected density, the
 * context's ranks r_d), and phi_ij = sum_t mu_t G_ij x_d (C_td U_d,ij) (Eq. final) with the
 * context's 1-D convolution matrices C_td (its quadrature); the context's shared bases are not
 * used.  W_i = - sum_j psi_j * phi_ij.  Arguments, layouts, aliasing rules and errors are those of
 * tx_exchange_apply; runs in float32 on the CUDA cores whatever the context's precision (the
 * eigenvectors from a Jacobi method in float32); TX_ERR_UNSUPPORTED_SHAPE for n_d > 160.  The
 * first call makes float32 copies of C_td (T n_d^2 floats per mode).
 */
int tx_exchange_apply_sthosvd(tx_ctx* ctx, const float* psi_occ, int n_occ, const float* psi_tgt, int n_tgt,
                              float* out, tx_stream_t stream);

/*
 * tx_set_quadrature -- how the 1-D convolution integrals are evaluated (Eqs. quadVal, discInteg).
 *   order 0             nodal quadrature with the context's weights (the default):
 *                       C_td[a][b] = w_b exp(-theta_t (x_a - x_b)^2)
 *   order p in 1..8     finite-element quadrature: the 1-D field is interpolated by Lagrange
 *                       elements of order p (element e holds nodes p e .. p e + p; n_d - 1 must be a
 *                       multiple of p) and every element is integrated with `points` (1..64)
 *                       Gauss-Legendre points:
 *                       C_td[a][b] = sum_{e holds b} sum_q J_e w_q N_b(x_q) exp(-theta_t (x_a - x_q)^2)
 * A_td = C_td U_d is recomputed in float64 on the device (mu_t folded into mode 3) and the operand
 * copies of the context's precision are rebuilt.  The energy and the other inner products keep
 * the context's weights.  Synchronises the context's last stream.  TX_ERR_INVALID_ARG for an
 * order or point count out of range, TX_ERR_SHAPE if n_d - 1 is not a multiple of the order.
 */
int tx_set_quadrature(tx_ctx* ctx, int order, int points, tx_stream_t stream);

/*
 * Transfer of orbitals between an unstructured finite-element basis and the structured grid of
 * a context (section "Transfer of wavefunctions", Eq. interpolate):
 *     psi_s[i][a] = sum_b N_ab psi_u[b][i]
 * N_ab being the value at structured node a of the shape function of node b of the unstructured
 * cell that contains a.  The map (which structured nodes lie in which cell, and their N rows) is
 * computed once by tx_transfer_create and stored on the device; each transfer is then one
 * batched per-cell product over all orbitals.  The reverse transfer interpolates the structured
 * field (tensor-product Lagrange elements of order_s on the grid nodes) at every unstructured
 * node.
 *
 * tx_transfer_create: ctx gives the structured grid (its nodes and device).  X: host float64
 *   [n_nodes][3] node coordinates of the unstructured mesh; conn: host int32
 *   [n_cells][(order_u + 1)^3] global node of each local node (lx, ly, lz) at index
 *   (lx (order_u + 1) + ly) (order_u + 1) + lz; every cell is an axis-aligned box with its local
 *   nodes on a tensor product of 1-D node sets (the Lagrange nodes may sit anywhere inside
 *   it; the mesh may be refined with hanging nodes).  Where several cells contain a structured
 *   node (a shared face) the cell listed first gives its value.  order_s: order of the
 *   structured elements along every axis (n_d - 1 must be a multiple).  Orders 1 to 3.  The
 *   inputs are copied; the transfer keeps no pointer to them nor to ctx.  Synchronous.
 *   Errors: TX_ERR_INVALID_ARG (NULL or empty mesh, orders outside 1..3, a node index out of
 *   range), TX_ERR_NOT_SETUP (bad ctx), TX_ERR_SHAPE (n_d - 1 not a multiple of order_s, or
 *   structured nodes outside every cell), TX_ERR_OOM.
 * tx_transfer_u_to_s: psi_u device float32 [n_nodes][n_orb] (orbital index fastest, as an FE code
 *   stores them) -> psi_s device float32 [n_orb][n1][n2][n3].  Asynchronous on stream.
 * tx_transfer_s_to_u: psi_s [n_orb][n1][n2][n3] -> psi_u [n_nodes][n_orb].  Asynchronous.
 * tx_transfer_map_bytes: device bytes of the stored map (0 for a bad handle).
 * tx_transfer_destroy: frees the map (NULL is a no-op); the caller orders it after the
 *   transfers that use it.
 */
typedef struct tx_transfer tx_transfer;
int tx_transfer_create(tx_transfer** out, tx_ctx* ctx, int order_s, const double* X, int n_nodes, const int* conn,
                       int n_cells, int order_u);
int tx_transfer_u_to_s(tx_transfer* tr, const float* psi_u, int n_orb, float* psi_s, tx_stream_t stream);
int tx_transfer_s_to_u(tx_transfer* tr, const float* psi_s, int n_orb, float* psi_u, tx_stream_t stream);
long tx_transfer_map_bytes(const tx_transfer* tr);
void tx_transfer_destroy(tx_transfer* tr);

/* Release every device allocation of the context (after synchronising its last stream). */
void tx_destroy(tx_ctx* ctx);

/* Change the GEMM arithmetic of an existing context (operand copies are rebuilt). */
int tx_set_precision(tx_ctx* ctx, int precision, tx_stream_t stream);

/*
 * tx_exchange_apply -- out = K psi_tgt (Eqs. ExchangeOperator / hadam): for every target i,
 *   out_i = - sum_{j < n_occ} psi_occ_j * phi_ij.
 *   psi_occ   device float32 [n_occ][n1][n2][n3]
 *   psi_tgt   device float32 [n_tgt][n1][n2][n3]; NULL means the targets are psi_occ
 *             itself (n_tgt must then equal n_occ).  If psi_tgt points inside psi_occ at an
 *             orbital boundary, the targets are that slice of the occupied block and each
 *             pair potential shared by two targets is computed once (phi_ij = phi_ji).
 *   out       device float32 [n_tgt][n1][n2][n3], overwritten
 */
int tx_exchange_apply(tx_ctx* ctx, const float* psi_occ, int n_occ,
                      const float* psi_tgt, int n_tgt, float* out, tx_stream_t stream);

/*
 * tx_exchange_apply_energy -- out = K psi_occ and E_x = 1/2 sum_i <psi_i, out_i>_w in one
 * pass (the energy sums are taken in the same epilogue as the Hadamard products).
 *   out    device float32 [n_occ][n1][n2][n3], overwritten
 *   e_dev  device float64 scalar
 */
int tx_exchange_apply_energy(tx_ctx* ctx, const float* psi_occ, int n_occ, float* out, double* e_dev,
                             tx_stream_t stream);

/*
 * tx_exchange_energy -- E_x = 1/2 sum_i <psi_i, W_i>_w = -1/2 sum_ij sum_r w rho_ij phi_ij
 * (the exchange term of S[phi] with alpha = 1).  Writes one float64 to e_dev (device).
 * No W is stored: the weighted pair sums are reduced in float64 in a fixed order.
 */
int tx_exchange_energy(tx_ctx* ctx, const float* psi_occ, int n_occ, double* e_dev,
                       tx_stream_t stream);

/*
 * tx_exchange_energy_grad -- E_x and its gradient with respect to the nodal orbital values
 * (not in the paper; derived): with L = sum_t mu_t (x)_d A_td U_d^T,
 *   dE/dpsi_k = w * W_k - sum_j psi_j * L^T (w * rho_kj).
 *   grad   device float32 [n_occ][n1][n2][n3], overwritten
 *   e_dev  device float64 scalar, or NULL
 */
int tx_exchange_energy_grad(tx_ctx* ctx, const float* psi_occ, int n_occ, float* grad,
                            double* e_dev, tx_stream_t stream);

/*
 * tx_exchange_apply_vjp -- vector-Jacobian product of tx_exchange_apply for a cotangent
 * grad_out = dF/dout (plain sum over grid points):
 *   grad_tgt_k = - sum_j psi_j * L^T(grad_out_k * psi_j)
 *   grad_occ_j = - sum_k grad_out_k * phi_kj - sum_k psi_k * L^T(grad_out_k * psi_j)
 * psi_tgt must be a separate target block here (autograd adds the two gradients when the
 * caller's target and occupied tensors are the same).  grad_occ / grad_tgt are overwritten;
 * either may be NULL to skip it.
 */
int tx_exchange_apply_vjp(tx_ctx* ctx, const float* psi_occ, int n_occ,
                          const float* psi_tgt, int n_tgt, const float* grad_out,
                          float* grad_occ, float* grad_tgt, tx_stream_t stream);

/*
 * Batched application over many independent systems (grids, ranks and term counts may all
 * differ; no counterpart in the paper, whose MPI task grid distributes pairs of one system).
 * Each item is one tx_exchange_apply (e_dev NULL) or tx_exchange_apply_energy call (e_dev set,
 * psi_tgt NULL).  Items that share a context share its workspace and run one after another;
 * items with different contexts run concurrently on internal streams.
 */
typedef struct tx_batch_item {
    tx_ctx* ctx;
    const float* psi_occ;
    int n_occ;
    const float* psi_tgt;    /* NULL: targets are psi_occ */
    int n_tgt;
    float* out;              /* [n_tgt or n_occ][n1][n2][n3] */
    double* e_dev;           /* optional energy (requires psi_tgt == NULL) */
} tx_batch_item;
typedef struct tx_plan tx_plan;

/*
 * tx_batch_plan -- validates the items, reserves every workspace, and picks the expansion tile
 * plan of each distinct (n, r, T, precision).  tune_table: path of a text table of tuned plans
 * (read if it exists; when `autotune` is non-zero, shapes missing from it are timed on the
 * device with the items' own data and appended).  NULL: built-in heuristic only.  Runs one
 * untimed launch of every item (so later launches allocate nothing and can be captured).
 */
int tx_batch_plan(tx_plan** plan, const tx_batch_item* items, int n_items, const char* tune_table, int autotune,
                  tx_stream_t stream);

/* Enqueues every item on `stream` (fork / join through internal streams and events). */
int tx_batch_launch(tx_plan* plan, tx_stream_t stream);

/* Captures one tx_batch_launch into a CUDA graph owned by the plan (replaces any earlier one). */
int tx_batch_capture(tx_plan* plan, tx_stream_t stream);

/* Replays the captured graph on `stream` (one cudaGraphLaunch). */
int tx_batch_replay(tx_plan* plan, tx_stream_t stream);

/* Number of items and the expansion tile plan chosen for item i (x planes per CTA, stages). */
int tx_batch_item_plan(const tx_plan* plan, int i, int* bx, int* nstage);

void tx_plan_destroy(tx_plan* plan);

/* Forces the expansion tile plan of a context: bx x planes per CTA (1..16) and nstage operand
 * load stages (1..6); 0, 0 restores the built-in choice.  Returns TX_ERR_INVALID_ARG outside
 * those ranges and TX_ERR_UNSUPPORTED_SHAPE if the plan does not fit SMEM / TMEM. */
int tx_set_tile_plan(tx_ctx* ctx, int bx, int nstage);

/* Split precisions (TF32x3, BF16x3): phi = sum_t mu_t G x_d A_td (the final contraction of the
 * expansion, Eq. final) is accumulated on the tensor core for `terms` Gaussian terms at a time
 * and then added into a float32 accumulator held in registers (round to nearest).  The tensor
 * core rounds its float32 accumulator toward zero after every MMA, so the error grows with the
 * length of each tensor-core chunk; the hi*hi and the cross products (hi*lo + lo*hi) are
 * accumulated separately.  0 restores the default (1 term, the most accurate).  No effect on the
 * single-pass precisions.  TX_ERR_INVALID_ARG if < 0. */
int tx_set_accumulation_chunk(tx_ctx* ctx, int terms);

/* Single-pass precisions (BF16, TF32): form of the expansion kernel (the final contraction of
 * Eq. final, fused with the Hadamard product and the sum over j).  0 (default): automatic --
 * the persistent form, in which one CTA per SM walks the (pair, x slab) work items (one item per
 * 128-row y tile where a plane has more rows) and the epilogue of one item overlaps the MMAs of
 * the next, wherever its limits hold (at most two x planes per CTA, energy factors equal to the
 * multipliers); one CTA per work item elsewhere.  Stage 3 reads the stage-2 output Y from TMEM
 * as a TF32 operand.  Where a plane's last y tile is short (at most 64 rows), the persistent form
 * packs the last tiles of several planes into one 128-row item: their stage-2 products go to
 * disjoint TMEM lanes of one stage-2 buffer (the stage-2 operand of each plane is a zero-padded
 * window of A_t2), so stage 3 runs once for all of them instead of once per plane.  1: always
 * one CTA per work item.  2 (bf16 only): a persistent form in which converter warps round Y to
 * bf16 into shared memory so that stage 3 also runs as bf16 (measured slower than form 0 on the
 * Pt- and TiO2-shaped blocks: the extra hop lengthens the per-term chain of barriers).  3: form 0
 * without the packing of short y tiles.  4 (bf16 only, where r3 rounded up to 8 is a multiple of
 * 32 and an item holds at most two planes): form 0 with Y rounded to bf16 in place in TMEM by
 * two groups of converter warps, so that stage 3 runs as a bf16 MMA with A read from TMEM; phi is
 * double-buffered in TMEM and read by a four-warp epilogue (measured 10% slower than form 0 on
 * the TiO2-shaped block).  5 (bf16 only, at most two planes per item, T >= 2): form 0 with two
 * warps issuing the stage-2 MMAs and two the stage-3 MMAs, each pair taking alternate Gaussian
 * terms (the stage-3 pair hands a token back and forth so that phi accumulates in term order);
 * phi is double-buffered in TMEM and read in place by eight epilogue warps (measured 2% faster
 * than form 0 on a 64 x 32 cut of the TiO2-shaped block and equal on the whole block, slower on
 * the Pt-shaped one, where the second phi buffer leaves room for one plane per item, not two).  All forms give the same result up to
 * float32 summation order (forms 2 and 4 up to the bf16 rounding of Y).  TX_ERR_INVALID_ARG
 * outside 0..5. */
int tx_set_expansion_form(tx_ctx* ctx, int form);

/* Host-only description of the expansion kernel (the final contraction of Eq. final with the
 * Hadamard product and the sum over j, the dominant kernel) that tx_exchange_apply and
 * tx_exchange_apply_energy launch for a context of this shape, precision and expansion form
 * (0 to 5, as tx_set_expansion_form) with the built-in tile plan.  Needs no device and no
 * context.  n[3], r[3]: grid sizes and Tucker ranks; T: Gaussian terms.  Writes min(nout, 14)
 * values to out:
 *   [0] kernel: 0 float32 CUDA cores, 1 converter kernel (split precisions), 2 one CTA per
 *       (pair, x slab) item, 3 persistent (one CTA per SM walks the items), 4 persistent with
 *       stage 3 in bf16 from shared memory (form 2), 5 persistent with stage 3 in bf16 from
 *       TMEM (form 4), 6 persistent with two MMA-issuing warps per stage (form 5)
 *   [1] x planes per item   [2] stage-2 load stages   [3] stage-3 load stages (kernels 1-3)
 *   [4] stage-2 output buffers in TMEM (kernels 2, 3)   [5] TMEM columns allocated
 *   [6] dynamic shared memory bytes   [7] threads per CTA   [8] MMA K steps of stage 2
 *   [9] MMA K steps of stage 3   [10] n3 padded to 16   [11] items per pair (x slabs, times y
 *   tiles where an item covers one y tile; with packed last y tiles, the full tiles plus one item
 *   per group of packed planes; converter kernel with z parts: planes x y tiles x z parts)
 *   [12] planes whose last y tiles share one item (0: not packed)   [13] converter kernel: parts
 *   of the z columns, one per item, where a whole plane's phi does not fit (then one plane and
 *   one 128-row y tile per item, and [10] is the columns of one part; 0: whole planes)
 * For the float32 precision every value is 0.  Returns TX_OK; TX_ERR_INVALID_ARG for NULL
 * arrays, nout < 1, T < 1 or a form outside 0..5; TX_ERR_SHAPE for sizes outside
 * 2 <= n_d <= 4096, 1 <= r_d <= n_d; TX_ERR_UNSUPPORTED_PRECISION; TX_ERR_UNSUPPORTED_SHAPE
 * where tx_set_precision would refuse the shape. */
int tx_describe_expansion_plan(const int n[3], const int r[3], int T, int precision, int form, int* out, int nout);

/*
 * tx_exchange_apply_static -- out = K psi_occ (targets = the occupied block), like
 * tx_exchange_apply with psi_tgt NULL, for callers that cannot let a library allocate device
 * memory: code that gives all device memory to its own arena or pool allocator, or loops that
 * cannot afford the device-wide synchronisation cudaMalloc / cudaFree may cause.  The paper has
 * no counterpart; this is an interface of this library.
 *   - Allocates nothing (no cudaMalloc / cudaFree, no allocating library routine).  All scratch
 *     (pair table, projection and expansion intermediates) lives in one fixed 32 MiB array in
 *     the library's device memory, reserved on every device that loads the library until the
 *     process exits.  Sizes whose scratch for a single pair exceeds it are rejected with
 *     TX_ERR_UNSUPPORTED_SHAPE and a message giving the bytes needed.
 *   - Always runs the float32 kernels, whatever the context's precision.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current; make that first call before any stream capture.
 *   - Every call shares the array and leaves its contents behind; nothing in it is read before
 *     the same call writes it.  Calls whose GPU work overlaps (different streams, or different
 *     host threads on one device) race on the array: order them.
 *   psi_occ / out: device float32 [n_occ][n1][n2][n3]; out is overwritten.
 */
int tx_exchange_apply_static(tx_ctx* ctx, const float* psi_occ, int n_occ, float* out, tx_stream_t stream);

/*
 * Adaptively compressed exchange, the step after the exchange potentials ("ACE implementation"
 * section, Eqs. ace1 and eta).  With W_j = K psi_j (Eq. ace1: tx_exchange_apply of the occupied
 * block onto itself) and M_ij = <psi_i, W_j>_w (the grid's quadrature weights), the ACE operator is
 * V_ACE = - sum_k xi_k xi_k^T with xi_k = sum_i (L^-1)_ki W_i and -M = L L^T (Cholesky).
 *
 * tx_ace_projectors -- xi from psi_occ and W.
 *   psi_occ, W   device float32 [n_occ][n1][n2][n3] (W = K psi_occ, in any precision)
 *   xi           device float32 [n_occ][n1][n2][n3], overwritten (must not overlap the inputs)
 *   M            device float64 [n_occ][n_occ], receives M_ij = <psi_i, W_j>_w as computed; or NULL
 * M is formed with float32 products summed in float64; at a truncated Tucker rank it is slightly
 * asymmetric (the paper is silent on this), and its symmetric part (M + M^T) / 2 is factorised in
 * float64.  1 <= n_occ <= 4096.  The call synchronises `stream` to read the factorisation's outcome:
 * TX_ERR_NOT_DEFINITE if the symmetric part of M is not negative definite (xi is then invalid).
 * Scratch comes from the context's workspace (it may grow).
 */
int tx_ace_projectors(tx_ctx* ctx, const float* psi_occ, int n_occ, const float* W, float* xi, double* M,
                      tx_stream_t stream);

/*
 * tx_ace_apply -- out_a = V_ACE psi_a = - sum_k xi_k <xi_k, psi_a>_w for a block of n orbitals
 * (Eq. eta applied to a block).
 *   xi    device float32 [n_xi][n1][n2][n3] (from tx_ace_projectors)
 *   psi   device float32 [n][n1][n2][n3];  out  device float32 [n][n1][n2][n3], overwritten
 * Asynchronous; scratch from the context's workspace.
 */
int tx_ace_apply(tx_ctx* ctx, const float* xi, int n_xi, const float* psi, int n, float* out, tx_stream_t stream);

/* Size in bytes of the device workspace the context currently holds. */
size_t tx_workspace_bytes(const tx_ctx* ctx);

/* Upper bound on the workspace (default 2 GiB); larger calls are split into pair batches. */
int tx_set_workspace_limit(tx_ctx* ctx, size_t bytes);

/* Reads and clears the device-side error word (bounded waits that gave up, and best-effort
 * drains of in-flight copies that gave up); synchronises the context's last stream.  Returns
 * TX_OK or TX_ERR_TIMEOUT (the message names the wait that gave up). */
int tx_check_device_error(tx_ctx* ctx);

/* Time limit of every bounded device-side wait in this context's kernels (no counterpart in the
 * paper): a wait that has not completed after `ns` nanoseconds gives up, records where, and its
 * kernel unwinds (releasing its TMEM) so that the context stays usable; the host sees
 * TX_ERR_TIMEOUT from tx_check_device_error.  0 restores the default of 2 s.  Synchronises the
 * context's last stream.  TX_ERR_INVALID_ARG outside 1 us .. 60 s. */
int tx_set_wait_limit(tx_ctx* ctx, uint64_t ns);

/* Self-test of the bounded wait (no counterpart in the paper): launches one warp on `stream` that
 * (if hold_tmem != 0) allocates 32 TMEM columns and then waits on an mbarrier that nothing ever
 * completes.  After the context's wait limit the wait gives up exactly as a pipeline kernel's
 * would: it records the timeout in the context's error word, frees its TMEM and returns.  A
 * following tx_check_device_error returns TX_ERR_TIMEOUT and clears the word; the context then
 * works as before.  Nothing faults or hangs. */
int tx_selftest_wait(tx_ctx* ctx, int hold_tmem, tx_stream_t stream);

/*
 * tx_exchange_energy_from_w -- E = 1/2 sum_i sum_r w(r) psi_i(r) W_i(r) for given orbitals and
 * their exchange potentials W_i = K psi_i (the exchange term of S[phi] with alpha = 1, summed
 * over the n orbitals given).  Used to add up the energy of a target block applied on its own
 * (for instance one shard of the targets): the shards' values add up to E_x.
 *   psi, W  device float32 [n][n1][n2][n3];  e_dev  device float64 scalar
 * Reduced in float64 in a fixed order (deterministic).
 */
int tx_exchange_energy_from_w(tx_ctx* ctx, const float* psi, const float* W, int n, double* e_dev,
                              tx_stream_t stream);

/*
 * Self-check of the tensor-core GEMM building block used by every tensor-core precision (no
 * counterpart in the paper): D[b][m][n] = sum_k A[b][m][k] B[b][n][k] for device float32
 * A [batch][M][K], B [batch][N][K] (K a multiple of 8) rounded to the operand type of
 * `precision` (split into hi + lo for the 3-pass precisions), D float32 [batch][M][N].
 * Synchronises `stream`; allocates and frees its own scratch.
 */
int tx_selftest_gemm(int precision, int batch, int M, int N, int K, const float* A, const float* B, float* D,
                     tx_stream_t stream);

const char* tx_status_string(int status);
const char* tx_last_error_message(void);

/*
 * Opt-in device timing of the library's own kernels: while enabled, each launch on the calling
 * thread is bracketed by CUDA events on its stream.  tx_profile_read synchronises those events
 * and returns, for the kernel class `name` ("project", "expand_mode1", "consume", "adjoint",
 * "gemm", ...), the number of launches and their summed device time in milliseconds.
 */
void tx_profile_enable(int enable);
void tx_profile_reset(void);
int tx_profile_read(const char* name, int* launches, double* total_ms);

/* Number of kernel launches this library made on the calling thread since the last reset. */
uint64_t tx_launch_count(void);
void tx_reset_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* TUXC_H */
