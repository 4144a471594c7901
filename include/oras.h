/*
 * oras.h -- C ABI of a single-GPU (GB300, sm_103a) solver for the linear systems that
 * degree-r Nedelec edge elements give for the time-harmonic Maxwell equations, solved by
 * flexible GMRES right-preconditioned with the Optimized Restricted Additive Schwarz
 * (ORAS) method.
 *
 * Paper: M. Bonazzoli, V. Dolean, F. Rapetti, P.-H. Tournier, "Parallel preconditioners
 * for high order discretizations arising from full system modeling for brain microwave
 * imaging", arXiv:1605.04521.
 *   Sec. 2  : curl-curl equation, impedance boundary condition, variational formulation.
 *   Sec. 3  : generators lambda^k w^e of degree r and their DOFs.
 *   Sec. 4  : M^{-1}_ORAS = sum_s R_s^T D_s A_s^{-1} R_s with impedance transmission.
 *   Sec. 5  : GMRES preconditioned by ORAS; pseudo-block treatment of many right-hand sides.
 *
 * Conventions shared by every entry point:
 *   - Complex numbers are interleaved (re, im) doubles: oras_complex is layout-compatible
 *     with C99 double _Complex and std::complex<double>.
 *   - Multi-vector arguments (rhs, x, v, z) are N x k column-major: vector j starts at
 *     offset j*N, N = oras_ndof(h).
 *   - `mem` selects where a data pointer lives: ORAS_MEM_HOST (pageable or pinned host
 *     memory) or ORAS_MEM_DEVICE (device memory of the current CUDA device, e.g. a torch
 *     tensor's data_ptr()).  Device pointers are read/written on the handle's stream.
 *   - The caller owns every buffer it passes; the library copies what it keeps.  The
 *     library owns all device memory it allocates and frees it in oras_destroy().  Device
 *     memory comes from the current device's default stream-ordered memory pool, whose
 *     release threshold the library sets to unlimited: freed memory stays in the pool and
 *     serves the next handle without mapping new pages.  oras_release_memory() returns it.
 *   - Return codes: 0 = ORAS_OK, > 0 = warning, < 0 = error.  Nothing throws across the
 *     ABI.  oras_last_error(h) (or oras_last_error(NULL) before a handle exists) gives a
 *     message for the last failing call on this thread.
 *   - Local numbering: the vertices of each tetrahedron are sorted by global id; the n_loc
 *     local DOFs are the 6 edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3) (r each), the 4 faces
 *     (0,1,2),(0,1,3),(0,2,3),(1,2,3) (r(r-1) each) and the volume (r(r-1)(r-2)/2).
 *     Global numbering: edge DOFs (edges sorted by vertex pair), then face DOFs (faces
 *     sorted by vertex triple), then volume DOFs (tetrahedron order).
 */
#ifndef ORAS_H
#define ORAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } oras_complex;

typedef struct oras_handle oras_handle;

enum {
  ORAS_OK = 0,
  ORAS_NOT_CONVERGED = 1,        /* x holds the best iterate of the last cycle           */
  ORAS_PENDING = 2,              /* serving: the request has not finished yet            */
  ORAS_ERR_INVALID_ARG = -1,
  ORAS_ERR_BAD_MESH = -2,        /* index out of range, repeated vertex, zero volume     */
  ORAS_ERR_OUT_OF_MEMORY = -3,
  ORAS_ERR_SINGULAR_LOCAL = -4,  /* a local matrix A_s had an exactly zero pivot column */
  ORAS_ERR_DEVICE_TIMEOUT = -5,  /* a bounded device-side wait gave up                   */
  ORAS_ERR_CUDA = -6,
  ORAS_ERR_REJECTED = -7,        /* request over the admission budget (serving)          */
  ORAS_ERR_UNSUPPORTED = -8,
  ORAS_ERR_STATE = -9            /* call order: e.g. solve before factor                 */
};

enum { ORAS_MEM_HOST = 0, ORAS_MEM_DEVICE = 1 };
enum { ORAS_WEIGHTS_POU = 0 /* ORAS: R_s^T D_s */, ORAS_WEIGHTS_NONE = 1 /* OAS, Sec. 4 */ };
enum { ORAS_OVERLAP_VERTEX = 0, ORAS_OVERLAP_FACE = 1 };
enum { ORAS_LU_AUTO = 0 /* tensor cores for FP32 factors */, ORAS_LU_CUDA_CORES = 1 };
/* Preconditioner apply with FP32 factors: AUTO streams the factor arena once per group of up to
 * 32 right-hand sides through tcgen05 tensor-core products (TF32 operands, FP32 accumulation)
 * when a call has 8 or more columns, and once per group of up to 4 on the CUDA cores (FP32)
 * otherwise; CUDA_CORES always takes the CUDA-core groups. */
enum { ORAS_APPLY_AUTO = 0, ORAS_APPLY_CUDA_CORES = 1 };
/* Transmission condition of the local problems (Sec. 4): impedance (ORAS: A_s = sum of the
 * element matrices of Omega_s^delta + i w~ S on its boundary faces) or Dirichlet (RAS:
 * A_s = R_s A R_s^T, the rows and columns N_s of the global matrix). */
enum { ORAS_TRANSMISSION_IMPEDANCE = 0, ORAS_TRANSMISSION_DIRICHLET = 1 };

/* Problem statement (Sec. 2-4).  All pointers are host pointers, read during the call. */
typedef struct {
  int64_t nv;                 /* number of vertices                                     */
  const double* xyz;          /* [nv][3] vertex coordinates                             */
  int64_t nt;                 /* number of tetrahedra                                   */
  const int32_t* tets;        /* [nt][4] vertex ids (any order; sorted internally)      */
  const oras_complex* eps_r;  /* [nt] relative permittivity, e^{i w t} convention:      */
                              /*      lossy media have Im(eps_r) < 0 (Sec. 2)            */
  const oras_complex* mu_r;   /* [nt] relative permeability, NULL -> 1                  */
  double k0;                  /* free-space wave number omega sqrt(eps0 mu0), mesh units */
  int32_t r;                  /* polynomial degree of the edge elements, 1..3 (Sec. 3)  */
  int32_t nsub;               /* number of subdomains N_sub (Sec. 4)                    */
  int32_t overlap;            /* overlap layers delta >= 0                              */
  const int32_t* part;        /* [nt] subdomain of each tetrahedron, or NULL for        */
                              /*      recursive coordinate bisection into nsub parts    */
  const double* beta_face;    /* [nt][4] impedance coefficient beta > 0 of Sec. 2 on the   */
                              /*   face of tetrahedron t opposite its vertex tets[4t+q]    */
                              /*   (the caller's vertex order); read for outer boundary    */
                              /*   faces only (other entries are ignored), kept for every  */
                              /*   later oras_factor of the handle.  NULL: beta = k0       */
                              /*   sqrt(Re mu_r Re eps_r) of the adjacent tetrahedron,     */
                              /*   from the materials of each oras_factor                  */
  const uint8_t* face_kind;   /* [nt][4] boundary condition on the same faces as beta_face: */
                              /*   ORAS_FACE_IMPEDANCE (0) or ORAS_FACE_METALLIC (1, E x n  */
                              /*   = 0 on Gamma_w, Sec. 2 eq. metallicbc; outer faces only).*/
                              /*   NULL: every outer face is an impedance face              */
} oras_problem;

/* Boundary condition of an outer face (oras_problem.face_kind).  On metallic faces the
 * degrees of freedom whose basis functions have a nonzero tangential trace there (those of the
 * face's edges and of the face) are constrained to zero: their rows and columns of A and of
 * every A_s become identity rows and columns, right-hand sides are zero there (oras_solve zeroes
 * them), and beta_face is not read for those faces. */
enum { ORAS_FACE_IMPEDANCE = 0, ORAS_FACE_METALLIC = 1 };

/* Solver options.  Zero-initialised fields take the defaults given in brackets. */
typedef struct {
  int32_t restart;            /* FGMRES restart length m [50]                           */
  int32_t max_iter;           /* total Arnoldi steps per right-hand side [5000]         */
  int32_t factor_bits;        /* 32: complex FP32 local factors; 64: complex FP64 [32]  */
  int32_t weights;            /* ORAS_WEIGHTS_POU [default] or ORAS_WEIGHTS_NONE        */
  int32_t overlap_kind;       /* ORAS_OVERLAP_VERTEX [default] or ORAS_OVERLAP_FACE     */
  int32_t lu_engine;          /* ORAS_LU_AUTO [default]: trailing updates of FP32 factors */
                              /*   on tcgen05 tensor cores (TF32 inputs, FP32 accumulate);*/
                              /*   ORAS_LU_CUDA_CORES: FP32 CUDA-core updates             */
  int32_t lu_panel;           /* outer LU panel width in 64-column tiles [8]: the trailing */
                              /*   matrix is updated once per panel                        */
  int32_t lu_group;           /* tensor-core update: 128-row output blocks per raster group  */
                              /*   (operand reuse in L2) [8]                                 */
  int32_t transmission;       /* ORAS_TRANSMISSION_IMPEDANCE [default] or _DIRICHLET (RAS) */
  int32_t graphs;             /* 1: run each Arnoldi step (apply, SpMV, orthogonalisation) as */
                              /*   a captured CUDA graph, captured on its second use and      */
                              /*   replayed afterwards; needs a non-default stream            */
                              /*   (oras_set_stream) and timing off [0]                       */
  int32_t wait_ms;            /* limit of every bounded device-side wait, in milliseconds: a  */
                              /*   wait on another warp or CTA that lasts longer gives up, the */
                              /*   kernel returns and the call reports ORAS_ERR_DEVICE_TIMEOUT */
                              /*   [2000]; waits of a CTA for its own copies in flight before  */
                              /*   it exits never use less than 2000                           */
  int32_t apply_engine;       /* ORAS_APPLY_AUTO [default] or ORAS_APPLY_CUDA_CORES            */
  int32_t block;              /* 1: oras_solve treats its k > 1 columns as one block (block      */
                              /*   flexible GMRES, Sec. 6); 0: k independent recurrences that   */
                              /*   share every kernel launch (pseudo-block, Sec. 5) [0]         */
  int32_t recycle;            /* k > 0: one-column oras_solve runs GCRO-DR(restart, k) and keeps */
                              /*   its deflation subspace in the handle for the next solve (Sec. */
                              /*   6, recycling across the imaging loop's systems) [0]          */
  int32_t reserved[2];
} oras_options;

/* Per right-hand-side outcome of oras_solve. */
typedef struct {
  int32_t iterations;         /* Arnoldi steps taken                                    */
  int32_t restarts;           /* completed FGMRES cycles                                */
  int32_t converged;          /* 1 if the true relative residual <= tol                 */
  int32_t pad;
  double relres;              /* true FP64 ||b - A x|| / ||b|| of the returned x        */
} oras_info;

/* Message of the last failing call on this thread for h (NULL: calls without a handle).  No
 * counterpart in the paper (error reporting).  Never fails; the string stays valid until the
 * next failing call on h or its destruction. */
const char* oras_last_error(const oras_handle* h);

/* Eigenvalues w[n] and unit eigenvectors V (row-major n x n, column j for w[j]; NULL allowed) of
 * the dense complex matrix A (row-major n x n, host): the QR algorithm the recycling solver uses
 * for its harmonic Ritz problems, exported for tests.  No counterpart in the paper.  Returns OK,
 * INVALID_ARG (n < 1, NULL A or w) or NOT_CONVERGED. */
int oras_dense_eig(int32_t n, const oras_complex* A, oras_complex* w, oras_complex* V);

/* Drops the deflation subspace that GCRO-DR solves (oras_options.recycle) keep in the handle, so
 * that the next solve starts without recycling.  INVALID_ARG for a NULL handle. */
int oras_recycle_reset(oras_handle* h);

/* Version of the ABI described here.  No counterpart in the paper.  Never fails. */
int32_t oras_abi_version(void);  /* 3: oras_problem.face_kind, ports (2: beta_face, wait_ms) */

/* ---------------------------------------------------------------- set-up */

/* Integer set-up of Sec. 3-4 on the host, no device work: sorted tetrahedra, edge and
 * face tables, global DOF numbering, outer boundary faces, partition (given or recursive
 * coordinate bisection), overlapping sets Omega_s^delta, ordered unknown sets N_s (Sec. 4,
 * R_s), Boolean partition of unity D_s (sum_s R_s^T D_s R_s = I), interface faces and the
 * CSR pattern of A.  p->eps_r, p->mu_r, p->k0 are ignored here.
 * Errors: INVALID_ARG (r not in 1..3, nsub < 1 or > nt, overlap < 0, NULL arrays, a
 * beta_face entry of an outer impedance face that is not finite and > 0, a face_kind entry
 * that is not 0 or 1, or 1 on an interior face),
 * BAD_MESH (vertex id out of range, repeated vertex, zero-volume tetrahedron, part entry
 * out of range), UNSUPPORTED (more than 2^31-1 DOFs or 2^21 vertices). */
int oras_create(const oras_problem* p, const oras_options* o, oras_handle** out);

/* Numeric set-up on the GPU for one material set (Sec. 2-4): element matrices
 *   A_T = mu_r^{-1} int curl w_a . curl w_b - k0^2 eps_r int w_a . w_b      (FP64, exact)
 * plus i beta int (w_a x n).(w_b x n) on outer faces, beta from oras_problem.beta_face or else
 * k0 sqrt(Re mu_r Re eps_r) of the adjacent tetrahedron; global CSR matrix A; dense local matrices A_s with impedance
 * transmission i omega~ on interface faces (omega~ from the tetrahedron inside Omega_s);
 * batched LU with pivoting of every A_s in the factor precision.  eps_r, mu_r: [nt] arrays
 * in `mem` (mu_r may be NULL -> 1).  May be called again with new materials (the mesh,
 * partition and device buffers are reused).  Errors: STATE, OUT_OF_MEMORY, CUDA,
 * SINGULAR_LOCAL, DEVICE_TIMEOUT. */
int oras_factor(oras_handle* h, const oras_complex* eps_r, const oras_complex* mu_r, double k0,
                int32_t mem);

/* oras_create followed by oras_factor(p->eps_r, p->mu_r, p->k0, ORAS_MEM_HOST) (Sec. 2-4).
 * Errors: those of oras_create and oras_factor; on failure nothing is kept and *out is
 * not set. */
int oras_setup(const oras_problem* p, const oras_options* o, oras_handle** out);

/* Frees host and device memory of h (NULL is ignored).  The device memory goes back to the
 * device's memory pool (see the conventions above).  No counterpart in the paper. */
void oras_destroy(oras_handle* h);

/* Returns to the driver the device memory that the default memory pool of `device` holds
 * unused (after oras_destroy), after synchronising that device.  No counterpart in the paper:
 * memory management of the single-GPU library.  Errors: INVALID_ARG (no such device), CUDA. */
int oras_release_memory(int32_t device);

/* Stream for all device work of h (a cudaStream_t; NULL = legacy default stream).  When the
 * largest subdomains get four CTAs in the preconditioner apply, their part runs on a side stream
 * that the handle owns, after an event recorded on h's stream and joined back into it by another
 * event, so all of h's work stays in the order of h's stream (stream capture included).  No
 * counterpart in the paper.  Errors: INVALID_ARG (h NULL). */
int oras_set_stream(oras_handle* h, void* stream);

/* ---------------------------------------------------------------- solve (Sec. 5) */

/* Solves A x_j = b_j for the k columns of rhs by FGMRES(m), x0 = 0, right-preconditioned
 * by ORAS, with FP64 Arnoldi (modified Gram-Schmidt), FP64 Givens rotations and an FP64
 * true-residual check at the end of every cycle; the k recurrences run together (pseudo-
 * block, Sec. 5).  With oras_options.block and k > 1: block FGMRES (Sec. 6 Block GMRES): one
 * block Krylov space for all k columns, FP64 block modified Gram-Schmidt between blocks, each new
 * block orthonormalised by CholQR2, the block least-squares problem kept triangular by
 * Householder reflections; info[j].iterations then counts block steps.  A block that becomes
 * numerically rank deficient (CholQR2 breakdown) ends the solve with ORAS_NOT_CONVERGED and the
 * last iterate.  With oras_options.recycle = r > 0 and k = 1: GCRO-DR(restart, r) (Sec. 6
 * subspace recycling; Parks, de Sturler et al. 2006) on A M^{-1}: deflated restarting with the
 * r harmonic Ritz vectors of smallest harmonic Ritz value, FP64 Gram-Schmidt against the
 * recycled C and the Arnoldi basis, and the deflation subspace kept in the handle for the next
 * solve (after an oras_factor with new materials it is recycled: C rebuilt from A M^{-1} U with r
 * products); info[0].iterations then counts the products with A M^{-1} (Arnoldi steps and the r
 * products that rebuild C).  Entries of the right-hand sides at unknowns constrained by metallic
 * faces are taken as zero.  rhs, x: N x k column-major in `mem`; info: k host structs or NULL.
 * Returns ORAS_OK when every column reached ||b - A x|| / ||b|| <= tol,
 * ORAS_NOT_CONVERGED when max_iter ran out for some column.  Errors: STATE (no
 * oras_factor yet), INVALID_ARG (k < 1 or > 64, tol <= 0), CUDA, OUT_OF_MEMORY,
 * DEVICE_TIMEOUT (a bounded device wait gave up during an Arnoldi step: the device status is
 * read after every step, and the solve stops there; x is not written). */
int oras_solve(oras_handle* h, const oras_complex* rhs, int32_t k, double tol, oras_complex* x,
               oras_info* info, int32_t mem);

/* ---------------------------------------------------------------- right-hand sides */

/* Impedance data of Sec. 2 for the plane wave E = p exp(-i gamma d.x),
 * gamma = k0 sqrt(mu_r eps_r) (principal root), on every outer face:
 * g = mu_r^{-1} (curl E) x n + i beta n x (E x n),  b_a = int_boundary g . w_a, with the
 * face's beta of oras_factor (oras_problem.beta_face or the derived one).
 * d: unit direction [3], p: polarisation [3] (host).  b: N values in `mem`.
 * Errors: INVALID_ARG (NULL arguments), STATE (no oras_factor yet), CUDA. */
int oras_rhs_plane_wave(oras_handle* h, const double* d, const oras_complex* p, oras_complex* b,
                        int32_t mem);

/* Point dipole: b_a = w_a(x0) . dir in the lowest-index tetrahedron whose barycentric
 * coordinates of x0 are all >= -1e-12.  x0, dir: [3] host.  b: N values in `mem`.  The
 * paper's sources are waveguide ports (Sec. 2); the point dipole is the synthetic source that
 * stands in for them.  Errors: INVALID_ARG (NULL arguments, or x0 in no tetrahedron), STATE
 * (no oras_factor yet), CUDA. */
int oras_rhs_dipole(oras_handle* h, const double* x0, const double* dir, oras_complex* b,
                    int32_t mem);

/* ---------------------------------------------------------------- waveguide ports (Sec. 2, 5)
 * A rectangular port on the outer boundary: the rectangle {origin + s u + t v : s, t in
 * [0, 1]}, u and v orthogonal, lying in the plane of the outer faces it covers.  Its faces are
 * the outer faces whose centroid ((x0 + x1) + x2) / 3 (vertices in ascending id order) lies in
 * the rectangle: 0 <= s, t <= 1 and distance to its plane at most 1e-9 (|u| + |v|).  Its
 * fundamental TE10 mode is E0(x) = sin(pi s) v / |v|, s = (x - origin) . u / |u|^2; beta > 0 is
 * the propagation wavenumber along the waveguide (give the same beta to the port's faces in
 * oras_problem.beta_face for the Silver-Mueller condition of eq. wgi).  Face integrals use the
 * collapsed Gauss-Legendre product rule with 12 x 12 points per face. */
typedef struct {
  double origin[3];
  double u[3];                /* width edge: the mode varies as sin(pi s) along it          */
  double v[3];                /* height edge: the mode points along it                      */
  double beta;                /* propagation wavenumber along the waveguide (> 0)          */
} oras_port;

/* Port vector p_a = int_port w_a . E0 (N values, real parts; imaginary parts zero) and its
 * norm N = int_port |E0|^2.  p: N values in `mem`; norm: host (NULL allowed).
 * Errors: INVALID_ARG (NULL arguments, u or v zero or not orthogonal to 1e-12, beta <= 0, no
 * outer face in the port), STATE (no oras_factor yet), CUDA. */
int oras_port_vector(oras_handle* h, const oras_port* port, oras_complex* p, double* norm, int32_t mem);

/* Load of a transmitting port (Sec. 2 eq. wgj): the incoming TE10 mode E_in = E0 exp(i beta
 * zeta) (zeta along the outward normal n, so the wave travels into the domain) gives the data
 * g = mu_r^{-1} (curl E_in) x n + i beta n x (E_in x n) = i beta (1 + 1/mu_r) E0 on the port,
 * and b_a = int_port g . w_a (mu_r of the face's tetrahedron; constrained entries zero).
 * b: N values in `mem`.  Errors: as oras_port_vector. */
int oras_rhs_port(oras_handle* h, const oras_port* port, oras_complex* b, int32_t mem);

/* Scattering coefficients (Sec. 5.1 eq. sij) of k fields at nports ports:
 *   S[i * k + j] = int_{port i} conj(E_j) . E0_i / int_{port i} |E0_i|^2
 *              = sum_a conj(x[a + j N]) p_i[a] / N_i,
 * x: the fields (N x k column-major in `mem`, e.g. oras_solve's output); on the transmitting
 * port the total field is used, as the formula is printed.  S: host [nports][k].  Sums in a
 * fixed order on the device.  Errors: as oras_port_vector, INVALID_ARG (k or nports < 1). */
int oras_s_matrix(oras_handle* h, int32_t nports, const oras_port* ports, const oras_complex* x, int32_t k,
                  oras_complex* S, int32_t mem);

/* Relative error of Sec. 5.2 (eq. errsij): sqrt(sum |S - S_ref|^2) / sqrt(sum |S_ref|^2) over
 * n entries (host arrays).  Returns -1 for NULL arrays, n < 1 or a zero S_ref. */
double oras_s_error(const oras_complex* S, const oras_complex* S_ref, int64_t n);

/* ---------------------------------------------------------------- queries (host data)
 * The mesh, numbering and subdomain data of oras_create (Sec. 3-4), copied to the caller's
 * host arrays.  Counts return -1 for a NULL handle; the int-returning calls return
 * INVALID_ARG for a NULL handle or output, or s out of range. */

int64_t oras_ndof(const oras_handle* h);            /* N, or -1                          */
int32_t oras_nlocal(const oras_handle* h);          /* n_loc = r(r+2)(r+3)/2, or -1      */
int32_t oras_nsub(const oras_handle* h);            /* N_sub, or -1                      */
/* out: [nt][n_loc] global DOF ids (local numbering in the header comment). */
int oras_dofmap(const oras_handle* h, int32_t* out);
/* out: [N] 1 for the degrees of freedom constrained by metallic faces, else 0. */
int oras_constrained_dofs(const oras_handle* h, uint8_t* out);
/* out: [nt] non-overlapping subdomain of each tetrahedron. */
int oras_partition(const oras_handle* h, int32_t* out);
/* Sizes of subdomain s: #N_s, #Omega_s^delta tetrahedra, padded factor order. */
int oras_subdomain_size(const oras_handle* h, int32_t s, int64_t* ndof, int64_t* ntet,
                        int64_t* npad);
/* dofs: [#N_s] ascending global ids of N_s (R_s); pou: [#N_s] D_s diagonal (0/1) or NULL;
 * tets: [#Omega_s^delta] ascending tetrahedron ids or NULL. */
int oras_subdomain(const oras_handle* h, int32_t s, int32_t* dofs, uint8_t* pou, int32_t* tets);
/* Number of stored nonzeros of A. */
int64_t oras_nnz(const oras_handle* h);
/* Bytes of the local-factor arena (device), 0 before oras_factor. */
int64_t oras_arena_bytes(const oras_handle* h);

/* ---------------------------------------------------------------- operator access */

/* Element matrices A_T (without boundary-face terms, Sec. 2-3) of `count` tetrahedra `tets`
 * (host), copied from the device into out[count][n_loc][n_loc] (host).  Errors: INVALID_ARG
 * (NULL arrays, tetrahedron id out of range), STATE (no oras_factor yet), CUDA. */
int oras_element_matrices(oras_handle* h, const int32_t* tets, int64_t count, oras_complex* out);
/* CSR of the global matrix A (Sec. 2-3; host arrays): rowptr [N+1], cols [nnz], vals [nnz];
 * any may be NULL.  Errors: INVALID_ARG (h NULL), STATE (vals before oras_factor), CUDA. */
int oras_global_csr(oras_handle* h, int64_t* rowptr, int32_t* cols, oras_complex* vals);
/* y = A x for k columns (N x k column-major, `mem`), the product of Sec. 5's GMRES.
 * Errors: INVALID_ARG (NULL vectors, k < 1 or > 64), STATE (no oras_factor yet),
 * OUT_OF_MEMORY, CUDA. */
int oras_matvec(oras_handle* h, const oras_complex* x, oras_complex* y, int32_t k, int32_t mem);
/* y = A x for k columns of complex FP32 x (N x k column-major pairs of floats, `mem`) into
 * complex FP64 y (N x k column-major): the product FGMRES forms with the preconditioned vectors
 * of FP32 factors.  Computed on the FP32 pipes with error-free transformations (A split into
 * FP32 hi + lo parts, exact product and sum errors carried), about 2^-48 relative error per
 * entry: the SpMV of Sec. 5's GMRES, formed on the FP32 pipes because GB300's FP64 pipe is
 * narrow.  Requires oras_factor.  Errors: INVALID_ARG, STATE, CUDA. */
int oras_matvec_c64(oras_handle* h, const void* x, oras_complex* y, int32_t k, int32_t mem);
/* z = M^{-1}_ORAS v for k columns (N x k column-major, `mem`), Sec. 4 (M^{-1}_OAS with
 * weights ORAS_WEIGHTS_NONE).  Synchronises the handle's stream before it returns.  Errors:
 * INVALID_ARG (NULL vectors, k < 1 or > 64), STATE (no oras_factor yet), OUT_OF_MEMORY, CUDA,
 * DEVICE_TIMEOUT (a bounded device wait of the apply gave up; z is not valid). */
int oras_precond(oras_handle* h, const oras_complex* v, oras_complex* z, int32_t k, int32_t mem);

/* Allocation-free preconditioner apply: z = M^{-1}_ORAS v for k columns, the same result as
 * oras_precond, for callers that must not allocate device memory during the call -- a serving
 * process whose device memory is entirely pre-reserved by a pool allocator (a raw cudaMalloc
 * would fail or fragment the pool), or a latency-bound loop where cudaMalloc/cudaFree would
 * synchronise the device and stall the other requests in flight.  The paper has no counterpart;
 * this is an interface convenience.  v, z: device pointers (current device = the handle's
 * device), N x k column-major, complex FP64, on the handle's stream; the call is asynchronous.
 * The local vectors live in one fixed 16 MiB device array compiled into the library (every GPU
 * that loads the library holds it until exit); sum over subdomains of the padded order times
 * the factor entry size (8 B FP32, 16 B FP64) must fit, else INVALID_ARG with the needed size.
 * The first call on a device resolves the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  Every call shares the array and leaves its last
 * contents there; each call writes every entry before reading it.  Calls that overlap on the
 * GPU (other streams, other threads) race on the array.  Nothing is allocated or freed.  Cost:
 * the k columns go through the apply one after the other, so the factor arena is streamed k
 * times (oras_precond streams it once per group of up to 4 columns with FP32 factors).  The call
 * does not wait for the GPU, so a bounded device wait that gives up inside it is not reported
 * (the kernel stops the affected subdomain and returns; z is then not valid).
 * Errors: INVALID_ARG (NULL vector, k < 1 or > 64, or the scratch need above 16 MiB: checked
 * from the host set-up alone, before the STATE check), STATE (no oras_factor yet), CUDA. */
int oras_precond_noalloc(oras_handle* h, const oras_complex* v, oras_complex* z, int32_t k);

/* Self-test of failure detection (no counterpart in the paper): runs, on the handle's stream,
 * one kernel that waits with each bounded-wait primitive of the library's kernels (a CTA-scope
 * mbarrier phase, a cluster-scope acquire on an mbarrier, a shared-memory counter) on a
 * condition that nothing ever satisfies, with the handle's limit oras_options.wait_ms.  Each
 * wait gives up, records the timeout in the handle's device status, and the kernel returns;
 * the call reads the status like oras_solve does and returns ORAS_ERR_DEVICE_TIMEOUT, with
 * detail (or NULL) = bit mask of the primitives that gave up (1 CTA mbarrier, 2 cluster
 * mbarrier, 4 counter; 7 when all behave).  The status is cleared again before returning, so the
 * handle stays usable.  Takes about 3 x wait_ms.  Errors: INVALID_ARG, STATE (no oras_factor
 * yet), CUDA. */
int oras_wait_selftest(oras_handle* h, int32_t* detail);

/* Autotuner of the batched LU's tile shapes (no counterpart in the paper): the outer panel width
 * (tiles of 64 columns per trailing update; trades the updates inside a panel against the passes
 * over the trailing matrix) and the raster group of the tensor-core update (output blocks that
 * share operands in L2).  Factorises the handle's current problem (materials of the last
 * oras_factor, on the handle's stream) once per candidate width 4, 8, 12, 16, 24, 32, 48, 64, 96,
 * 128, 192 (group 8), then once per group 16, 32, 64 at the best width, keeps the fastest pair in the
 * handle's options (lu_panel, lu_group) and leaves the factors of that pair.  The choice is
 * cached for the process under the problem's shape (factor precision, LU engine, padded
 * subdomain orders): a later handle of the same shape takes it without timing.  panel: chosen
 * width (or NULL); ms[0..nms): the candidates' factorisation times in milliseconds, widths then
 * groups (14 entries; -1 when taken from the cache; NULL allowed).
 * Errors: INVALID_ARG, STATE (no oras_factor yet), and those of oras_factor. */
int oras_autotune(oras_handle* h, int32_t* panel, double* ms, int32_t nms);
/* The raster group oras_autotune chose for the handle (0 before tuning: the default); -1 for
 * a NULL handle.  No counterpart in the paper (a tile shape of the batched LU). */
int32_t oras_lu_group(const oras_handle* h);

/* Device bytes that oras_factor followed by an oras_solve of k right-hand sides allocate for
 * this handle (factor arena, inverted diagonal blocks, A, element matrices, Krylov basis of
 * restart+1 FP64 and restart FP32/FP64 vectors per right-hand side, staging), including the
 * allocator's rounding.  Host-only: valid right after oras_create.  No counterpart in the
 * paper (admission control of the serving runtime).  Errors: INVALID_ARG. */
int oras_footprint(const oras_handle* h, int32_t k, int64_t* bytes);

/* ---------------------------------------------------------------- serving
 * Continuous batching of solve requests on one GPU (the imaging loop of Sec. 6 needs one
 * Maxwell solve per antenna and per permittivity update).  Requests of different meshes,
 * degrees and right-hand-side counts are accepted at any time.  Host threads run the mesh
 * set-up of each request (as oras_create), which fixes its device footprint (oras_footprint);
 * the oldest planned request is admitted as soon as a worker slot is free and its footprint
 * fits in the HBM budget beside the requests already on the GPU.  Each admitted request runs
 * assembly, batched LU and FGMRES on its slot's own CUDA stream, so the work of concurrent
 * requests overlaps on the device; its factors and Krylov basis stay resident until it
 * finishes.  Every result equals what oras_setup + oras_solve give for that request alone.
 * The paper has no serving interface; this is the library's. */
typedef struct oras_server oras_server;

typedef struct {
  int64_t hbm_budget;         /* device bytes the admitted requests may hold together;     */
                              /*   0: 90% of the device's free memory at creation          */
  int32_t device;             /* CUDA device ordinal [0]                                   */
  int32_t max_active;         /* requests on the GPU at once: worker threads, one CUDA     */
                              /*   stream each [4], at most 64                             */
  int32_t planners;           /* host threads for the set-up of queued requests [2]        */
  int32_t reserved[5];
} oras_server_config;

/* Life of one request; times in seconds since oras_server_create. */
typedef struct {
  double submit_s;            /* oras_submit returned                                      */
  double planned_s;           /* host set-up done, footprint known                         */
  double admitted_s;          /* admitted onto the GPU (0 if never)                        */
  double done_s;              /* result ready                                              */
  int64_t footprint;          /* device bytes reserved for it                              */
  int64_t ndof;               /* N of its problem (0 if set-up failed)                     */
  int32_t k;                  /* right-hand sides                                          */
  int32_t status;             /* its return code; ORAS_PENDING while unfinished            */
} oras_ticket;

typedef struct {
  int64_t hbm_budget, hbm_in_use, hbm_peak;   /* bytes                                     */
  int32_t queued;             /* submitted, not yet admitted                               */
  int32_t active;             /* on the GPU now                                            */
  int32_t peak_active;        /* most requests on the GPU at once so far                   */
  int32_t completed;          /* finished (any status but REJECTED)                        */
  int32_t rejected;           /* footprint above the whole budget                          */
  int32_t pad;
} oras_server_counters;

/* Starts the planner and worker threads (no GPU work until a request is admitted).
 * cfg may be NULL (defaults).  Errors: INVALID_ARG, CUDA (budget 0 and no device),
 * OUT_OF_MEMORY. */
int oras_server_create(const oras_server_config* cfg, oras_server** out);
/* Queues one solve: problem p and options o (NULL: defaults) as for oras_setup, and k
 * right-hand sides given either as rhs (host, n x k column-major, n = N of the problem) or
 * as dipoles (host, [k][6]: position x0 and direction of each point dipole, as
 * oras_rhs_dipole) -- exactly one of the two.  All inputs are copied before the call returns.
 * Returns a ticket > 0, or INVALID_ARG / OUT_OF_MEMORY / STATE (server shutting down).
 * Problems found later (bad mesh, n != N, footprint above the budget: REJECTED) are the
 * ticket's status. */
int64_t oras_submit(oras_server* srv, const oras_problem* p, const oras_options* o, const oras_complex* rhs,
                    int64_t n, const double* dipoles, int32_t k, double tol);
/* Waits up to timeout_ms (< 0: no limit) for the ticket.  Returns ORAS_PENDING if it is still
 * running (call again), else the request's status (as oras_solve's, or the error that stopped
 * it), copies the solution into x (host, n x k column-major, n = N; NULL: discard) and the
 * per-column outcome into info ([k] or NULL), and retires the ticket (oras_ticket_info keeps
 * its record).  Errors of the call itself: INVALID_ARG (unknown ticket; n != N for a solved
 * request, ticket kept), STATE (ticket already retired). */
int oras_wait(oras_server* srv, int64_t ticket, oras_complex* x, int64_t n, oras_info* info, int32_t timeout_ms);
/* Waits up to timeout_ms (< 0: no limit) until the ticket has finished, without retiring it
 * (then oras_ticket_info gives N and the status).  Returns ORAS_OK (finished or retired),
 * ORAS_PENDING, or INVALID_ARG (unknown ticket). */
int oras_ticket_wait(oras_server* srv, int64_t ticket, int32_t timeout_ms);
/* Record of a ticket, pending or retired.  Errors: INVALID_ARG (unknown ticket). */
int oras_ticket_info(oras_server* srv, int64_t ticket, oras_ticket* out);
/* Message of a failed ticket ("" if none); ticket <= 0: the last failing server call.  Never
 * fails ("" for a NULL server or an unknown ticket). */
const char* oras_server_error(oras_server* srv, int64_t ticket);
/* Budget, occupancy and counters.  Errors: INVALID_ARG (NULL server or output). */
int oras_server_stats(oras_server* srv, oras_server_counters* out);
/* Cancels queued requests (status STATE), lets running ones finish, joins the threads and
 * frees everything, including tickets nobody collected.  NULL is ignored. */
void oras_server_destroy(oras_server* srv);

/* ---------------------------------------------------------------- instrumentation
 * No counterpart in the paper: measurement of the library's own kernels.  The int-returning
 * calls return INVALID_ARG for a NULL handle or output. */

/* Device time accumulated by kernel class since the last oras_reset_timings, measured with
 * CUDA event pairs on the handle's stream while timing is on: t[2c] = milliseconds and
 * t[2c+1] = kernel launches of class c, for c = 0 element and face matrices, 1 global CSR
 * values, 2 local matrices (incl. arena clear), 3 LU tournament pivoting, 4 LU row
 * interchanges and the final transposition of the U tiles, 5 LU triangular tile solves, 6 LU
 * trailing updates, 7 preconditioner apply, 8 SpMV of FP32-valued vectors (Arnoldi with FP32
 * factors), 9 orthogonalisation and Givens, 10 other, 11 SpMV of FP64 vectors (true residual;
 * Arnoldi with FP64 factors), 12 LU panel updates (the column a left-looking panel step brings
 * up to date and the step's pivot tile row; class 6 is then the trailing update after each
 * panel).  n: entries of t (26 covers all). */
int oras_timings(const oras_handle* h, double* t, int32_t n);
/* Zeroes the accumulators of oras_timings. */
int oras_reset_timings(oras_handle* h);
/* Enables (1) / disables (0) event timing (default 0: no events are recorded). */
int oras_set_timing(oras_handle* h, int32_t on);
/* Number of CUDA kernels this library has launched in this process (all handles). */
int64_t oras_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* ORAS_H */
