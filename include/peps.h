/*
 * peps.h -- C ABI of the GB300 (sm_103a) boundary-MPS PEPS environment library.
 *
 * The library computes approximate environments of finite PEPS with open
 * boundary conditions by the sandwich (boundary-MPS) contraction of
 * Lubasch, Cirac & Banuls, "Unifying Projected Entangled Pair States
 * contractions", and the local quantities that follow from them:
 *
 *   - the norm <psi|psi>                                     (Section 2, Fig. 2)
 *   - the environment of every site, in factored form        (Section 2: N_l, b_l)
 *   - local expectation values <O> = Tr(rho O)/Tr(rho)       (Section 5.3)
 *   - the same environments in the cluster scheme CU         (Section 5, 5.2, 5.3)
 *   - the distance of a cluster boundary from the full one   (Section 5.2, Fig. Fid)
 *   - the environments of an infinite PEPS by the CU         (Section 5.4)
 *   - the tensor update that consumes the environments: the gate's action
 *     refit by ALS on the reduced tensors, with the full environment (full
 *     update) or the cluster environment CU_delta         (Section 2; Section 5)
 *
 * Around these: recorded plans (CUDA graphs) with an autotuner, the learned
 * cluster closure (a small MLP trained on the GPU), profiling counters,
 * failure detection (iteration caps, bounded waits, host-side fault
 * injection), checkpoint / resume of env handles and closure training, and
 * one entry point that allocates no device memory (peps_cu0_noalloc).
 *
 * Every step runs in the library's CUDA kernels; there is no CPU fallback.
 * A call made without a usable CUDA device fails with PEPS_ECUDA.
 *
 * Conventions
 *   - Every call returns PEPS_OK (0) or one of the status codes below; no
 *     C++ exception crosses this boundary.  peps_last_error() returns a
 *     thread-local message for the last failing call on that thread.
 *   - The caller owns every input and output array.  The library owns env
 *     handles (device-resident); peps_env_free releases one and accepts NULL.
 *   - Calls are ordered on the CUDA stream passed as `cuda_stream`
 *     (a cudaStream_t; NULL means the legacy default stream).  Calls that
 *     return host values synchronise that stream before returning.
 *   - Calls on the same env handle, or any two calls that run at the same
 *     time on different threads, must be serialised by the caller.
 *
 * Tensor layout (C order):
 *   A[y][x][s][u][l][n][r]   y = row (0 at the top), x = column,
 *                            s = physical index (dimension d),
 *                            u, l, n, r = up, left, down, right virtual legs (D each).
 *   Open boundary conditions: a leg that points out of the lattice has
 *   dimension 1 (Section 2, footnote on OBC tensors); in the dense array it
 *   uses index 0 only and every other entry on it must be 0, otherwise the
 *   call fails with PEPS_EINVAL.  Every entry must be finite (PEPS_EINVAL).
 */
#ifndef PEPS_H
#define PEPS_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PEPS_OK         0
#define PEPS_EINVAL     1   /* bad argument, shape or OBC entries                    */
#define PEPS_ENOMEM     2   /* device allocation failed                              */
#define PEPS_ECUDA      3   /* CUDA runtime error, or no CUDA device                 */
#define PEPS_ECONVERGE  4   /* an iteration (Jacobi SVD, CU_0 fixed point) hit its cap */
#define PEPS_ETIMEOUT   5   /* a device-side bounded wait ran out                    */

/* element type of A */
#define PEPS_F64 0
#define PEPS_F32 1

/* compression of the boundary MPS after each absorbed row (Section 2) */
#define PEPS_SVD 0          /* QR sweep to canonical form, then SVD truncation to chi */
#define PEPS_VAR 1          /* one-site ALS sweeps, local equation N A = b with N = 1 */

/* arithmetic of the absorb contractions (tensor cores, FP32 accumulation);
 * QR, SVD, gauge fixing and rescaling are FP64 in every mode.  The X3 modes
 * split each operand into a rounded high part and a rounded residual and sum
 * the three leading products (hi*hi + hi*lo + lo*hi). */
#define PEPS_PREC_FP64   0
#define PEPS_PREC_TF32   1
#define PEPS_PREC_BF16   2
#define PEPS_PREC_TF32X3 3
#define PEPS_PREC_BF16X3 4

/* local quantity selectors */
#define PEPS_SITE  0        /* rho of site (y,x):            d x d,     Ly*Lx values       */
#define PEPS_HBOND 1        /* rho of bond (y,x)-(y,x+1):    d^2 x d^2, Ly*(Lx-1) values   */
#define PEPS_VBOND 2        /* rho of bond (y,x)-(y+1,x):    d^2 x d^2, (Ly-1)*Lx values   */

/* cluster closure outside the window */
#define PEPS_CLOSURE_PLAIN   0   /* CU_0 separable boundaries (Section 5.1)                 */
#define PEPS_CLOSURE_LEARNED 1   /* CU_0 matrices replaced by the learned closure's output   */
#define PEPS_CLOSURE_WIDTH   256 /* hidden width of the learned closure used by peps_env_cluster */

typedef struct {
    int Ly, Lx;          /* lattice size, >= 1 each                                   */
    int d;               /* physical dimension, 1..4                                  */
    int D;               /* virtual bond dimension, 1..16                             */
    int dtype;           /* PEPS_F64 or PEPS_F32                                      */
    const void* A;       /* dense tensors, layout above; read only                    */
    int on_device;       /* 1: A is a device pointer, 0: a host pointer               */
} peps_lattice;

typedef struct {
    int chi;             /* boundary bond dimension D' (>= 1)                          */
    int mode;            /* PEPS_SVD or PEPS_VAR                                       */
    int sweeps;          /* PEPS_VAR half-sweeps; <= 0 selects 2 (L->R then R->L)      */
    int precision;       /* PEPS_PREC_*                                                */
    int n;               /* cluster window edge length (peps_env_cluster), >= 1        */
    int closure;         /* PEPS_CLOSURE_PLAIN or PEPS_CLOSURE_LEARNED                 */
    const void* closure_weights;   /* LEARNED: device float* weights (width 256), see  */
                                   /* peps_mlp_param_count; else ignored               */
    unsigned long long seed;       /* keys the counter-based noise of the var start    */
} peps_opts;

typedef struct peps_env peps_env;   /* opaque, device resident, library owned */

/*
 * peps_env_full -- full (sandwich) environments of every site.
 *   Section 2 (Fig. 2, "sandwich contraction"): the norm network is swept
 *   row by row from the top and from the bottom, and column by column from
 *   the left and the right; each row is absorbed into the boundary MPS
 *   (ket layer, then bra layer) and the result is compressed to bond chi.
 *   The environment of site l (Section 2) is then held in factored form
 *   (top and bottom boundary, left and right row environments), from which
 *   the reduced density matrices of every site, horizontal bond and
 *   vertical bond are formed.  Vertical bonds use the column sweeps.
 *   *out receives a new handle (set to NULL on failure).
 */
int peps_env_full(const peps_lattice* lat, const peps_opts* opts,
                  peps_env** out, void* cuda_stream);

/*
 * peps_env_cluster -- cluster (CU) environments of every site.
 *   Section 5 / 5.2: outside a window around each site the environment is
 *   the product of CU_0 separable boundaries (Section 5.1: D'=1 boundary
 *   found by ALS whose local solution is proportional to b_l); inside the
 *   window the contraction is the full one at bond chi.  Section 5.3 forms
 *   the cluster around the local term itself: the window is opts->n x
 *   opts->n with rows y-ceil(n/2)+1 .. (same for columns), clipped at the
 *   lattice edge, so edge windows are smaller.  Site (y,x) yields its own
 *   density matrix and those of the bonds to (y,x+1) and (y+1,x).  With
 *   n >= 2*max(Ly,Lx) every window is the lattice and the result equals
 *   peps_env_full's (Section 5: CU_{L-1} is the full update).
 *   Fails with PEPS_ECONVERGE if a CU_0 iteration does not converge.
 */
int peps_env_cluster(const peps_lattice* lat, const peps_opts* opts,
                     peps_env** out, void* cuda_stream);

/*
 * peps_env_cluster_range -- peps_env_cluster for the windows of the anchors
 *   with row-major index y*Lx + x in [anchor_begin, anchor_end).  The
 *   windows are independent (Section 5.2: separate processors each contract
 *   their own clusters and need only the small separable-boundary tensors),
 *   so a set of calls whose ranges partition [0, Ly*Lx) -- e.g. one per GPU
 *   -- yields every site's and bond's density matrix exactly once: the
 *   handle holds those of its own anchors (site (y,x), bonds to (y,x+1) and
 *   (y+1,x)) and zeros elsewhere.  The CU_0 boundaries are computed in full
 *   by every call.  0 <= anchor_begin <= anchor_end <= Ly*Lx, else PEPS_EINVAL.
 */
int peps_env_cluster_range(const peps_lattice* lat, const peps_opts* opts, long long anchor_begin,
                           long long anchor_end, peps_env** out, void* cuda_stream);

/*
 * peps_expect_local -- <O> = Tr(rho O) / Tr(rho) at every site or bond.
 *   Section 5.3 (local expectation values from local reduced density matrices).
 *   kind: PEPS_SITE / PEPS_HBOND / PEPS_VBOND.
 *   op:   host array, real, row-major, d x d (site) or d^2 x d^2 (bond, rows
 *         and columns ordered (s_first, s_second) with the first site the left
 *         or upper one); O[t][s] is <t|O|s>.
 *   out:  host array receiving Ly*Lx, Ly*(Lx-1) or (Ly-1)*Lx values in
 *         row-major order of the first site.
 *   lat:  may be NULL; if given its shape must match the env's.
 *   Synchronises the stream.
 */
int peps_expect_local(const peps_env* env, const peps_lattice* lat, int kind,
                      const double* op, double* out, void* cuda_stream);

/*
 * peps_env_rho -- copy the (unnormalised) reduced density matrices to the host.
 *   Same ordering as peps_expect_local; each entry is d x d (site) or
 *   d^2 x d^2 (bond) with rows = ket indices, columns = bra indices.
 *   out must hold count * d^2 (site) or count * d^4 (bond) doubles.
 *   Synchronises the stream.
 */
int peps_env_rho(const peps_env* env, int kind, double* out, void* cuda_stream);

/*
 * peps_norm -- ln |<psi|psi>| and its sign.
 *   Section 2: top-down sandwich sweep through the second-to-last row, then
 *   the last row contracted exactly against the last boundary.  Every
 *   boundary is rescaled to unit norm and the logs of the factors are
 *   accumulated, so the result does not overflow.  Synchronises the stream.
 */
int peps_norm(const peps_lattice* lat, const peps_opts* opts,
              double* ln_norm, int* sign, void* cuda_stream);

/*
 * peps_cu0_noalloc -- CU_0 separable boundaries without any device allocation.
 *   The paper has no counterpart: this is a service of the library.  It
 *   computes the same top-down separable (D'=1) boundaries that
 *   peps_env_cluster uses outside its windows, for callers that cannot call
 *   cudaMalloc -- e.g. a serving process whose own allocator already holds
 *   the device memory it may use, code in a latency-critical loop where
 *   cudaMalloc / cudaFree would synchronise the device, or a host framework
 *   that forbids device allocation after start-up.
 *   A:      device pointer, dense double [Ly][Lx][d][D][D][D][D] (layout and
 *           OBC rule as above; not validated here).
 *   sigma:  device pointer receiving double [Ly][Lx][D][D]: sigma[r][x] is
 *           the positive matrix on the (ket, bra) up legs of site (r, x), in
 *           the top-left du x du block (du = 1 on row 0, else D), zeros elsewhere;
 *           row 0 holds the trivial 1 x 1 closure.  Other directions: pass the
 *           lattice flipped or transposed.
 *   Limits: Ly <= 4096, Lx <= 64, d <= 4, D <= 8; larger sizes fail with
 *   PEPS_EINVAL.  Scratch is a file-scope device array of 65,608 doubles
 *   (about 513 KiB) that every GPU loading the library holds until exit.
 *   The first call on a device looks up that array's device address
 *   (cudaGetSymbolAddress); make the first call before any stream capture.
 *   Every call shares the array: two calls whose work overlaps on the GPU
 *   (different streams, or different host threads) race.  The call clears
 *   its status words itself.  Allocates nothing; synchronises the stream.
 *   Fails with PEPS_ECONVERGE if a cut needs more than 200 half-sweeps.
 *   Cost: the whole lattice runs on one 256-thread CTA (one SM), about
 *   Ly * Lx * h * 8 d D^5 FP64 flops for h half-sweeps per cut; at the
 *   largest sizes with slowly converging cuts a call can take many minutes.
 *   The Python binding checks rank, shapes, dtype (float64), contiguity and
 *   device of both tensors before calling, since the C side cannot.
 */
int peps_cu0_noalloc(const double* A, int Ly, int Lx, int d, int D, double* sigma,
                     void* cuda_stream);

/*
 * Learned cluster closure (the paper has no learned part; built on its
 * cluster scheme, Section 5.2).  A three-layer ReLU network of width W maps,
 * for one outward leg of a cluster window, the site tensor just above the
 * cut (d*D^4, zero-padded, legs [s,u,l,n,r] in the sweep's orientation),
 * the CU_0 matrix sigma0 at that leg (D^2) and its Cholesky factor L0 (D^2)
 * -- F = d*D^4 + 2*D^2 inputs -- to Y (D x D); the closure matrix is
 * X X^T / ||X X^T||_F with X = L0 + Y, positive, and sigma0 when Y = 0.
 * Weights (float32, device): W1[W][F] b1[W] W2[W][W] b2[W] W3[D^2][W] b3[D^2].
 * The matrix products run on the tensor cores in BF16 with FP32 accumulation.
 *
 * peps_closure_data: training examples of one lattice.  Runs the four full
 *   boundary sweeps at opts->chi and the CU_0 boundaries; for every
 *   orientation o (top-down, bottom-up, left-right, right-left), cut r >= 1
 *   and column x it writes the features (row of X, F floats) and the label
 *   (row of Y, D^2 floats): the site matrix of the best product (D'=1)
 *   approximation of the full boundary at that cut.  X, Y are device
 *   pointers; with both NULL only *count is set.  D <= 8.
 * peps_mlp_param_count: number of floats in the weight vector.
 * peps_mlp_init: He-uniform hidden layers, zero biases and zero output layer.
 * peps_mlp_loss_grad: mean over n of ||sigma - label||_F^2 and its gradient
 *   (device float*, same layout as the weights); loss returned on the host.
 * peps_mlp_train: AdamW (beta 0.9/0.999, eps 1e-8) on minibatches of `batch`
 *   examples drawn by a seeded shuffle per epoch; *final_loss = mean
 *   minibatch loss over the last min(steps, 20) steps.
 * peps_mlp_predict: closure matrices (n x D^2, device float*).
 * All synchronise the stream.
 */
int peps_closure_data(const peps_lattice* lat, const peps_opts* opts, float* X, float* Y,
                      long long capacity, long long* count, void* cuda_stream);
long long peps_mlp_param_count(int d, int D, int width);
int peps_mlp_init(float* w, int d, int D, int width, unsigned long long seed, void* cuda_stream);
int peps_mlp_loss_grad(const float* w, const float* X, const float* Y, long long n, int d, int D,
                       int width, double* loss, float* grad, void* cuda_stream);
int peps_mlp_train(float* w, const float* X, const float* Y, long long n, int d, int D, int width,
                   int steps, int batch, float lr, float weight_decay, unsigned long long seed,
                   double* final_loss, void* cuda_stream);
int peps_mlp_predict(const float* w, const float* X, long long n, int d, int D, int width,
                     float* sigma, void* cuda_stream);

/*
 * Checkpoint and resume (the paper keeps boundaries on disk or in memory,
 * Section 5.4; these calls make results and training state durable).
 * peps_mlp_train_state -- peps_mlp_train with the AdamW state held by the
 *   caller: adam_m, adam_v are device float* of peps_mlp_param_count each
 *   (zero them before the first call), *step (host) the steps already taken
 *   with them; on success *step += steps.  Bias correction and the seeded
 *   minibatch stream continue from *step, so a run split into calls with the
 *   same seed, n and batch gives the same weights as one call.
 * peps_mlp_save / peps_mlp_load -- weights (and, when adam_m / adam_v are
 *   non-NULL, the AdamW moments and *step) to / from a file: one JSON header
 *   line padded to 512 bytes ({"format":"peps-mlp", d, D, width, params,
 *   state, step}), then the float32 arrays.  Loading checks the shape; a file
 *   without optimizer state loads zero moments and step 0.  w, adam_m, adam_v
 *   are device pointers.
 * peps_env_save / peps_env_load -- an environment handle's results (the
 *   density matrices of every site and bond, ln|<psi|psi>| and its sign,
 *   the lattice shape) to / from a file: a 512-byte JSON header line
 *   ({"format":"peps-env", kind, Ly, Lx, d, D, has_norm, array sizes}), then
 *   the float64 arrays.  peps_env_load creates a new handle (free it with
 *   peps_env_free) that peps_expect_local, peps_env_rho and peps_env_ln_norm
 *   read like the original.  A file of another format, shape or size fails
 *   with PEPS_EINVAL; file errors with PEPS_EINVAL naming the path.
 *   All synchronise the stream.
 */
int peps_mlp_train_state(float* w, float* adam_m, float* adam_v, long long* step, const float* X, const float* Y,
                         long long n, int d, int D, int width, int steps, int batch, float lr, float weight_decay,
                         unsigned long long seed, double* final_loss, void* cuda_stream);
int peps_mlp_save(const char* path, const float* w, const float* adam_m, const float* adam_v, long long step, int d,
                  int D, int width, void* cuda_stream);
int peps_mlp_load(const char* path, float* w, float* adam_m, float* adam_v, long long* step, int d, int D, int width,
                  void* cuda_stream);
int peps_env_save(const peps_env* env, const char* path, void* cuda_stream);
int peps_env_load(const char* path, peps_env** out, void* cuda_stream);

/*
 * peps_ipeps_cluster -- local density matrices of an infinite PEPS by the
 *   cluster update's environment (Section 5.4: a CU procedure for iPEPS needs
 *   only the dominant D'=1 boundary eigenvector, O(dD^5), followed by a
 *   cluster contraction as in the finite case).  Single-site unit cell:
 *   every site holds A[s][u][l][n][r] (d x D^4, every leg D; host or device
 *   pointer per on_device).  For each side the separable boundary is the
 *   fixed point of the CU_0 update of an infinite row (Section 5.1) whose
 *   horizontal environments are the row's own left / right fixed points
 *   (identities to start, unit-norm matrices, converged when no matrix moves
 *   by 1e-13; PEPS_ECONVERGE after 25x the CU_0 half-sweep cap).  An
 *   opts->n x opts->n window of copies of A closed by those four boundaries
 *   (corners dropped) is then contracted at bond opts->chi as a finite window
 *   (mode, sweeps, precision, seed as in peps_env_cluster); the anchor sits
 *   at row and column ceil(n/2)-1.
 *   rho_site (d x d), rho_h (d^2 x d^2, the bond to the right), rho_v (d^2 x
 *   d^2, the bond below; zero when n = 1): host arrays, unnormalised, same
 *   index order as peps_env_rho.  sigma (host, may be NULL): the boundary
 *   matrices top, bottom, left, right, D x D each.  Synchronises the stream.
 */
int peps_ipeps_cluster(const double* A, int d, int D, int on_device, const peps_opts* opts, double* rho_site,
                       double* rho_h, double* rho_v, double* sigma, void* cuda_stream);

/*
 * Failure detection (the paper has no counterpart).
 *
 * peps_set_iteration_caps -- caps of the library's iterations: the
 *   half-sweeps of a CU_0 fixed point (Section 5.1; default 200) and the
 *   sweeps of a one-sided Jacobi SVD (svd mode; default 60).  A computation
 *   that reaches a cap fails with PEPS_ECONVERGE.  0 restores a default;
 *   values above 1e6 fail with PEPS_EINVAL.  Process-wide, for calls made
 *   afterwards; a recorded plan keeps the caps it was recorded with.  Needs
 *   no GPU.
 * peps_wait_selftest -- one kernel that spins on a device flag nothing sets,
 *   with the same bounded-wait shape as the library's device-side waits, for
 *   budget_us microseconds (1..1e6) of the GPU's global timer; it returns
 *   PEPS_ETIMEOUT through the device status word, and the context stays
 *   usable.  For tests of the timeout path.  Synchronises the stream.
 *
 * Host-side fault injection: the environment variable PEPS_FAULT, read at
 * the start of every call, forces an error path of that call without
 * touching the GPU's state:
 *   PEPS_FAULT=alloc     every device allocation of the call fails  -> PEPS_ENOMEM
 *   PEPS_FAULT=nan       a NaN is planted in the call's own device copy of the
 *                        lattice before its validation              -> PEPS_EINVAL
 *   PEPS_FAULT=converge  both iteration caps are 1 for the call     -> PEPS_ECONVERGE
 *                        (where an iteration does not stop after one step)
 * Inputs with non-finite entries fail with PEPS_EINVAL in every call that
 * takes a lattice.
 */
int peps_set_iteration_caps(int cu0_half_sweeps, int jacobi_sweeps);
int peps_wait_selftest(int budget_us, void* cuda_stream);

/*
 * peps_bond_update -- the tensor update of the full update (FU) for a set of
 *   bonds.  Section 2: after a Trotter gate acts on a bond, the two tensors
 *   of the bond are refit by alternating least squares, one tensor at a
 *   time, each solving N_l A_l = b_l; the unknowns are the reduced tensors
 *   (Section 2, footnote: O(D^6) linear systems).  Each site is split by a
 *   thin QR, left site as (u l n) x (s r), right site as (u n r) x (t l); N
 *   is the norm network with the two reduced tensors removed, contracted
 *   from the full (sandwich) environment at bond opts->chi.  Every bond of
 *   the call uses the environment of the input state -- the bonds of one
 *   Trotter set updated independently, the parallel scheme of Sections 4.4
 *   and 5.2.
 *   Rules where the paper is silent: N is symmetrised and replaced by its
 *   positive part; the ALS starts from the truncated SVD of the gated pair;
 *   each system is shifted by 1e-12 * trace / size and solved by Cholesky;
 *   the result is split by an SVD into U sqrt(S) | sqrt(S) V^T (largest entry
 *   of every U column positive), the new bond keeps min(D, k_l d, k_r d)
 *   values (zero beyond), and both new tensors are scaled to unit norm.
 *   lat:       device lattice (on_device = 1), F64 or F32, read only.
 *   opts:      chi, mode, sweeps, precision, seed of the environment
 *              (n, closure ignored).
 *   gate:      host, (d*d) x (d*d) row-major, G[(s t), (s' t')] with s the
 *              first site (left / upper) of every bond.
 *   bonds:     host, 3 * nbonds ints (kind, y, x): kind 0 the bond
 *              (y,x)-(y,x+1), kind 1 the bond (y,x)-(y+1,x); no site in two
 *              bonds (PEPS_EINVAL otherwise).
 *   als_iters: ALS rounds (each a left and a right solve), 1..1000.
 *   A_out:     device, the lattice's dtype and layout; may be lat->A (the
 *              update in place); sites outside the bonds are copied.
 *   cost:      host, nbonds doubles or NULL: |psi - G phi|^2_N / |G phi|^2_N
 *              of every bond after the fit.
 *   Needs d*D*D <= 160 (Cholesky systems in shared memory).  Synchronises
 *   the stream.
 */
int peps_bond_update(const peps_lattice* lat, const peps_opts* opts, const double* gate, const int* bonds,
                     int nbonds, int als_iters, void* A_out, double* cost, void* cuda_stream);

/*
 * peps_bond_update_cluster -- the same tensor update with the cluster
 *   update's environment, CU_delta.  Section 5: the cluster of size delta
 *   around a row is every row within distance delta of it (and likewise for
 *   columns); the environment of a horizontal bond in row y is the exact
 *   contraction (at bond opts->chi) of rows y-delta .. y+delta, clipped at the
 *   lattice edge, over all columns, closed above and below by the CU_0
 *   separable boundaries of those cuts (Section 5.1; at the lattice edge the
 *   lattice's own closures).  Vertical bonds use the column strip.  delta = 0
 *   is CU_0 (Section 5.1, a generalised simple update); delta >= L-1 is the
 *   full update.  Every bond of the call uses the CU_0 boundaries and clusters
 *   of the input state (the parallel CU of Section 5.4): one strip per row or
 *   column holding bonds, each with its own two sweeps of at most delta rows.
 *   Arguments, rules and errors as peps_bond_update; delta < 0 fails with
 *   PEPS_EINVAL; a CU_0 boundary that needs more than its half-sweep cap
 *   fails with PEPS_ECONVERGE.
 */
int peps_bond_update_cluster(const peps_lattice* lat, const peps_opts* opts, int delta, const double* gate,
                             const int* bonds, int nbonds, int als_iters, void* A_out, double* cost,
                             void* cuda_stream);

/*
 * peps_boundary_fidelity -- distance of a cluster environment from the full one.
 *   Section 5.2, Fig. Fid: the boundary MPS on the right legs of column 0
 *   (the environment of the left-most column) in the cluster form -- columns
 *   delta .. 1 absorbed at bond opts->chi into the CU_0 separable boundary
 *   (Section 5.1) of the columns right of column delta; delta >= Lx-1 is
 *   the full contraction (Section 2) -- against the full contraction at bond
 *   chi_ref.  *one_minus_f = 1 - f, f = |tr(rho_ref^T rho)| with both scaled
 *   to tr(rho^T rho) = 1.  opts->mode, sweeps, precision and seed apply to
 *   both contractions (var noise keyed by the rows of the absorbed part).
 *   Needs Lx >= 2; the overlaps are FP64.  Synchronises the stream.
 */
int peps_boundary_fidelity(const peps_lattice* lat, const peps_opts* opts, int delta, int chi_ref,
                           double* one_minus_f, void* cuda_stream);

/* peps_env_ln_norm -- the norm recorded in a full env (PEPS_EINVAL for cluster envs). */
int peps_env_ln_norm(const peps_env* env, double* ln_norm, int* sign, void* cuda_stream);

/* peps_env_free -- release a handle; NULL is accepted. Not stream ordered:
 * it synchronises the device work that used the handle first. */
void peps_env_free(peps_env* env);

/* peps_last_error -- message of the last failing call on this thread. */
const char* peps_last_error(void);

/*
 * Recorded plans.  The paper has no counterpart: a plan is the sweep of
 * peps_env_full (cluster = 0) or peps_env_cluster (cluster != 0) recorded
 * once as a CUDA graph and replayed, so that the thousands of small
 * launches of a call cost one graph launch.  Every bond dimension, window
 * and launch shape depends on the lattice shape and the options only, and
 * every data-dependent quantity (norms, log-scales, convergence) stays on
 * the device, so the recorded graph is valid for any tensor values.
 *
 * peps_plan_create: lat->A must be device memory (on_device = 1).  The call
 *   first runs the plain computation once (validating the input, including
 *   the OBC rule), then records.  The plan keeps lat->A's address and
 *   opts->closure_weights' address: the caller keeps both buffers alive and
 *   may overwrite their contents between runs (same shapes).  Records on an
 *   internal stream; must not overlap another library call on the same
 *   device.  *out is NULL on failure.
 * peps_plan_run: replays the whole computation on cuda_stream, then
 *   synchronises it and returns the status (PEPS_ECONVERGE, PEPS_ETIMEOUT,
 *   PEPS_EINVAL for a degenerate state, as the plain calls).
 * peps_plan_env: the plan's environment handle (owned by the plan, valid
 *   until peps_plan_free; its contents are those of the last run).  Use it
 *   with peps_expect_local, peps_env_rho, peps_env_ln_norm; never pass it to
 *   peps_env_free.
 * peps_plan_tune: as peps_plan_create, with the launch configuration chosen
 *   by measurement (a project-written autotuner).  It records one plan per
 *   candidate and times one warm plus two timed replays of each with CUDA
 *   events on cuda_stream, keeping the fastest.  The search is over host
 *   lanes {2, 4, 8} first (QR cluster size by the library's model), then,
 *   for the cluster scheme, over the windows per batched launch {8, 16, 32},
 *   then over the largest QR cluster {8, 4}.  *lanes and *qr_cluster (either
 *   may be NULL) receive the choice.  Costs five recordings (seven for the
 *   cluster scheme), each timed over three replays.
 * peps_plan_launches: kernel launches in one replay (the kernel nodes of the
 *   recorded graph; 0 for NULL).
 * peps_plan_free: synchronises the device, releases the graph and its
 *   memory; NULL is accepted.
 */
typedef struct peps_plan peps_plan;
int peps_plan_create(const peps_lattice* lat, const peps_opts* opts, int cluster, peps_plan** out,
                     void* cuda_stream);
int peps_plan_run(peps_plan* plan, void* cuda_stream);
int peps_plan_tune(const peps_lattice* lat, const peps_opts* opts, int cluster, peps_plan** out,
                   int* lanes, int* qr_cluster, void* cuda_stream);
const peps_env* peps_plan_env(const peps_plan* plan);
long long peps_plan_launches(const peps_plan* plan);
void peps_plan_free(peps_plan* plan);

/*
 * Instrumentation (library-wide, not per handle).
 *   peps_profile_enable(mask): bit i of mask enables timing of kernel class
 *   i -- a CUDA event pair is recorded around each launch of that class, on
 *   the stream the kernel runs on (0 disables, -1 enables every class).
 *   peps_profile_read sums the event intervals per class after synchronising
 *   them.  Classes are named by peps_profile_name(i) for i in
 *   [0, peps_profile_count()).  launches counts kernel launches whether or
 *   not timing is enabled; flops / bytes are algorithmic counts (formula,
 *   not hardware counters).  The counters are process-wide and not
 *   thread-safe against concurrent readers.
 *   Recorded plans: the classes enabled when a plan is recorded are timed
 *   inside every replay (the event pairs are recorded as external event
 *   nodes of the graph); each peps_plan_run adds the replay's launches,
 *   flops, bytes and those times to the counters.
 */
void        peps_profile_enable(int mask);
void        peps_profile_reset(void);
int         peps_profile_count(void);
const char* peps_profile_name(int cls);
int         peps_profile_read(int cls, long long* launches, double* ms,
                              double* flops, double* bytes);

#ifdef __cplusplus
}
#endif
#endif /* PEPS_H */
