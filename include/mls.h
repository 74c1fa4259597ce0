/*
 * mls.h -- C ABI of the GB300 moving-least-squares (MLS) transfer library.
 *
 * The library builds MLS shape functions for Lagrangian markers (centroids of
 * surface triangles) immersed in an Eulerian grid and uses them to move data
 * between the two meshes, following Section 2 of Spandan, Lohse, de Tullio &
 * Verzicco, "A fast moving least squares approximation with adaptive
 * Lagrangian mesh refinement for large scale immersed boundary simulations"
 * (J. Comput. Phys.; arXiv:1805.01113):
 *
 *   build      Phi^T(x_l) = p^T(x_l) A^-1(x_l) B(x_l)          Eqs. 3, 4, 6
 *              (exact-MLS), or the Shepard blend of tabulated
 *              exact shape functions                            Eqs. 9, 10
 *              plus the spreading scale c_l                      Eqs. 7, 8
 *   interpolate U_l = sum_k phi_k^l u_k                          text after Eq. 6
 *   spread      f_k += sum_l c_l phi_k^l F_l                     text after Eq. 7
 *
 * Conventions shared by every entry point
 *   - Every call returns an int status (MLS_OK = 0, codes below).  A non-zero
 *     code leaves outputs unspecified; mls_last_error() gives a message for the
 *     calling thread.
 *   - Pointers marked "device" point to CUDA device memory owned by the
 *     caller; the library never frees them.  Pointers marked "host" are read
 *     during the call only.  Handles (mls_ctx, mls_transfer) are owned by the
 *     library and released by their destroy call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on it unless stated otherwise; the
 *     caller orders its own reads of outputs after the stream.
 *   - "real" is the context's arithmetic type: double for MLS_F64, float for
 *     MLS_F32.  "field" is the storage type of Eulerian fields: double,
 *     float or bfloat16 (MLS_BF16).
 *   - Marker arrays are structure-of-arrays: x[3][M] (x, then y, then z), one
 *     row of M values per component; same for U and F.  Eulerian fields are
 *     u[3][nz][ny][nx], x fastest.
 *   - Support node order: k = 9*(a_z+1) + 3*(a_y+1) + (a_x+1) for offsets
 *     a in {-1,0,1}^3 around the home cell (the cell with
 *     face_i <= x < face_{i+1} on every axis).
 */
#ifndef MLS_GB300_H
#define MLS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define MLS_OK                0
#define MLS_ERR_INVALID_ARG   1  /* bad pointer, size, option or handle combination */
#define MLS_ERR_CAPACITY      2  /* more markers than the transfer handle was created for */
#define MLS_ERR_UNSUPPORTED   3  /* valid request this build does not implement */
#define MLS_ERR_CUDA          4  /* a CUDA runtime call failed (see mls_last_error) */
#define MLS_ERR_OUT_OF_DOMAIN 5  /* mls_transfer_status: some markers were dropped */

/* ---- methods and number types ---------------------------------------- */
#define MLS_EXACT     0  /* exact-MLS, Eqs. 3-6 */
#define MLS_FAST      1  /* fast-MLS, Eqs. 9-10 */
#define MLS_SURROGATE 2  /* learned surrogate of exact-MLS with exact fallback (not in the paper) */

#define MLS_F64  0
#define MLS_F32  1
#define MLS_BF16 2

typedef struct mls_ctx mls_ctx;
typedef struct mls_transfer mls_transfer;

/* Eulerian grid (Section 2, Fig. 1a): per-axis face coordinates.  Cell i of
 * axis d spans [faces[d][i], faces[d][i+1]); its centre is a support node and
 * its width enters Eqs. 7-8.  Axis order is x, y, z. */
typedef struct {
  int32_t n[3];              /* cells per axis, >= 3; n[0]*n[1]*n[2] < 2^31 */
  int32_t periodic[3];       /* 1: supports wrap around; 0: walled, a marker
                                whose support would leave the grid is dropped */
  const double* faces[3];    /* host, n[d]+1 strictly increasing values */
} mls_grid;

typedef struct {
  int32_t real;          /* MLS_F64 or MLS_F32 (default MLS_F32) */
  int32_t field;         /* MLS_F64 (needs real = MLS_F64), MLS_F32 or MLS_BF16 */
  double eps;            /* Gaussian weight W = exp(-r^2/eps^2), r in home-cell
                            widths per axis (reading of the text after Eq. 2); default 1 */
  int32_t n_sub;         /* fast-MLS sub-Eulerian points per axis (Fig. 1b/1c), 3..33, default 9 */
  int32_t brick_log2[3]; /* spreading tile of 2^b home cells per axis, 1..5 each, default 3 */
  double cond_max;       /* MLS_F32 only: re-solve Eq. 6 in double when cond_1(A) exceeds this; <= 0 disables; default 1e6 */
  int32_t refine;        /* MLS_F32 only: iterative-refinement steps of the solve, 0..2, default 1 */
  double residual_max;   /* MLS_SURROGATE: linear-reproduction residual above which a marker
                            falls back to exact-MLS, default 1e-4 */
  int32_t basis;         /* size m of the MLS basis p (Section 2, text after Eq. 2: Pascal's
                            pyramid): 4 = [1, x, y, z] (the paper's, default) or
                            10 = [1, x, y, z, x^2, y^2, z^2, xy, yz, zx].  MLS_EXACT and
                            MLS_FAST (whose table holds exact shape functions) take either;
                            the surrogate and mls_interpolate_gradient need 4 and return
                            MLS_ERR_UNSUPPORTED otherwise */
} mls_options;

/* Device views into a built transfer (borrowed; valid until the next build on
 * the handle or its destruction).  Markers are stored in "tile order", a
 * permutation of the caller's order that groups markers by spreading tile
 * and, inside a tile of at most 2^12 cells, by home cell (the order among
 * markers of one home cell is not fixed). */
typedef struct {
  int64_t M;             /* markers in the last build */
  const void* phi;       /* device, real[27][capacity]: phi[k][j] for stored marker j (Eq. 6 / Eq. 9) */
  const void* c;         /* device, real[capacity]: c_l of Eq. 8 (0 for dropped markers) */
  const int32_t* home;   /* device, int32[capacity]: (iz*ny + iy)*nx + ix of the home cell, -1 if dropped */
  const int32_t* perm;   /* device, int32[capacity]: caller's marker index of stored marker j */
  int64_t capacity;
} mls_transfer_arrays;

/* Device-side counters of the last build (read with mls_transfer_status). */
typedef struct {
  int64_t dropped;       /* markers outside the grid, non-finite, or with a support leaving a walled axis */
  int64_t nonfinite;     /* of which: non-finite position or area */
  int64_t refined_fp64;  /* MLS_F32 exact builds re-solved in double (cond_1(A) > cond_max) */
  int64_t surrogate_fallback; /* MLS_SURROGATE markers that took the exact-MLS value */
} mls_status;

typedef struct {
  const char* name;      /* kernel name (static string) */
  int64_t launches;
  double total_ms;       /* sum of CUDA-event durations on the launching stream */
} mls_kernel_time;

/* Fill `opt` with the defaults listed above.  Never fails for non-NULL opt. */
int mls_options_default(mls_options* opt);

/* Create a context for one grid and option set on the current CUDA device.
 * Copies the grid to the device (allocates; synchronous).  Fails with
 * MLS_ERR_INVALID_ARG on non-increasing faces, n < 3, or bad options, and
 * with MLS_ERR_UNSUPPORTED when fast-MLS tables would be needed for more than
 * one non-uniform axis (checked lazily at the first MLS_FAST build). */
int mls_create(const mls_grid* grid, const mls_options* opt, mls_ctx** out);
int mls_destroy(mls_ctx* ctx);

/* Allocate a transfer handle for up to `capacity` markers (synchronous
 * allocation of phi, c, home, perm and the tile-sort workspace).  Builds
 * into it allocate nothing. */
int mls_transfer_create(mls_ctx* ctx, int64_t capacity, mls_transfer** out);
int mls_transfer_destroy(mls_transfer* T);

/* Marker preparation (Section 3, Fig. 5a; Eq. 7): for triangle t with
 * vertices V1, V2, V3 = vertices[tri[t][0..2]], write the centroid
 * x[:, t] = ((V1 + V2) + V3)/3 and the area area[t] = |(V2-V1)x(V3-V1)|/2,
 * evaluated in the context's real type in exactly that operation order
 * (IEEE round-to-nearest, no contraction).
 *   vertices  device, real[n_vertices][3] (interleaved x, y, z)
 *   tri       device, int32[n_tri][3]
 *   x         device, real[3][n_tri]     area  device, real[n_tri]
 * A triangle with a vertex index outside [0, n_vertices) gets a NaN centroid
 * (the next build drops and counts it). */
int mls_marker_prep(mls_ctx* ctx, const void* vertices, int64_t n_vertices,
                    const int32_t* tri, int64_t n_tri, void* x, void* area, void* stream);

/* mls_marker_prep of triangles [t_begin, t_end) only: x[:, t] and area[t]
 * for t in that range, in the same arrays of n_tri markers (other entries
 * untouched).  A caller that uploads the vertices in pieces (bodies in
 * order, each body's triangles referring to its own vertices) can prepare
 * each piece's markers as soon as its vertices are on the device, while the
 * next piece is copied; only vertices that the range's triangles refer to
 * are read.
 * Errors: MLS_ERR_INVALID_ARG unless 0 <= t_begin <= t_end <= n_tri, on
 * negative sizes, and on NULL pointers with a non-empty range. */
int mls_marker_prep_range(mls_ctx* ctx, const void* vertices, int64_t n_vertices,
                          const int32_t* tri, int64_t n_tri, int64_t t_begin, int64_t t_end,
                          void* x, void* area, void* stream);

/* mls_marker_prep_range of triangles [t_begin, t_end) fused with the first
 * phase of the next build of T (Section 2: each marker's home cell and its
 * spreading tile, as the build does first): the kernel that forms a marker
 * also locates it, so x and area are written and not read back.  Pieces go
 * in order: a piece with t_begin = 0 starts a new marker set (it resets T's
 * counters and tile bins on `stream`), and every other piece must start
 * where the previous one on T ended, with the same n_tri, x and area.  The
 * next mls_build_transfer / mls_build_interpolate / mls_build_direct_forcing
 * on T with M = n_tri, the same x and area, and pieces covering [0, n_tri)
 * then skips its own locate pass; any other build locates its markers
 * itself, as without this call.  In between, T holds scratch: the counters
 * of mls_transfer_status count the pieces so far, and T's transfer
 * functions must not be used (mls_interpolate, mls_spread and the like on T
 * wait for the build).  x and area must not change before that build, and
 * the pieces and the build run in stream order (one stream, or the caller's
 * events between streams).
 *   vertices, tri, x, area: as mls_marker_prep (x real[3][n_tri], area real[n_tri])
 * Errors: MLS_ERR_CAPACITY if n_tri exceeds T's capacity; MLS_ERR_INVALID_ARG
 * on NULL handles or pointers, a transfer of another context, negative
 * sizes, a range outside [0, n_tri], or a piece that does not follow the
 * previous one. */
int mls_marker_prep_locate(mls_ctx* ctx, mls_transfer* T, const void* vertices, int64_t n_vertices,
                           const int32_t* tri, int64_t n_tri, int64_t t_begin, int64_t t_end,
                           void* x, void* area, void* stream);

/* Build the transfer functions of M markers into T (Section 2).
 *   x     device, real[3][M] marker positions; area device, real[M] (A_l, Eq. 7)
 *   method MLS_EXACT (Eqs. 3-6), MLS_FAST (Eqs. 9-10; the first fast build
 *          on a context tabulates exact shape functions on the sub-Eulerian
 *          mesh, once, on `stream`), or MLS_SURROGATE (needs trained or
 *          loaded parameters, else MLS_ERR_UNSUPPORTED).
 * Markers are sorted into spreading tiles; phi, c, home and perm are written
 * in that order (see mls_transfer_arrays).  Dropped markers get phi = 0,
 * c = 0, home = -1 and are counted in mls_status.
 * Errors: MLS_ERR_CAPACITY if M > capacity; MLS_ERR_INVALID_ARG on NULL
 * pointers with M > 0 or an unknown method. */
int mls_build_transfer(mls_ctx* ctx, mls_transfer* T, const void* x, const void* area,
                       int64_t M, int32_t method, void* stream);

/* Euler-to-Lagrange interpolation U_l = sum_k phi_k^l u_k (text after Eq. 6)
 * for the 3 components, accumulated in the real type.
 *   u  device, field[3][nz][ny][nx]     U  device, real[3][M] (caller's marker order)
 * Dropped markers get U = 0. */
int mls_interpolate(mls_ctx* ctx, const mls_transfer* T, const void* u, void* U, void* stream);

/* mls_build_transfer followed by mls_interpolate of the same markers
 * (Section 2: Eqs. 3-6, then U_l = sum_k phi_k^l u_k, text after Eq. 6), in
 * one call: the order of an immersed-boundary step, whose markers move before
 * the velocity is interpolated to them.  For MLS_EXACT with the linear basis
 * the interpolation is done inside the build kernel, each phi_k multiplied
 * with the field at its node as it is formed (phi, c, home and perm are still
 * written to T for a later spread), so the field is read once and phi is not
 * read back; other methods and bases run the two calls in turn.  Arguments,
 * outputs and errors are those of the two calls; the results equal theirs up
 * to the rounding order of the sums (dropped markers get U = 0).
 *   u  device, field[3][nz][ny][nx]     U  device, real[3][M] (caller's marker order) */
int mls_build_interpolate(mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M,
                          int32_t method, const void* u, void* U, void* stream);

/* Gradients of an interpolated field at the markers (Section 2: MLS also
 * approximates spatial derivatives, which the solver needs for velocity and
 * pressure gradients at the markers): G[c][d][l] = sum_k d_d phi_k^l u_c,k,
 * with d_d phi the derivative of the exact-MLS shape functions (Eq. 6) with
 * respect to the marker position, the support and home cell of the last
 * build of T held fixed.  With gamma = A^-1 p(x_l):
 *   d_d phi_k = d_d W_k p_k.gamma + W_k p_k.A^-1 (d_d p - d_d A gamma).
 * The shape-function derivatives are formed on the fly (not stored), for
 * every method T was built with.
 *   x  device, real[3][M] the marker positions given to mls_build_transfer
 *   u  device, field[3][nz][ny][nx]      G  device, real[3][3][M] (component,
 *      direction, caller's marker order)
 * Dropped markers get G = 0. */
int mls_interpolate_gradient(mls_ctx* ctx, const mls_transfer* T, const void* x, const void* u, void* G,
                             void* stream);

/* Lagrange-to-Euler spreading f_k += sum_l c_l phi_k^l F_l (text after
 * Eq. 7).  Accumulates into f (the caller zeroes it when it wants a fresh
 * field); partial sums are formed per spreading tile in the real type and
 * added to f with atomic adds, so the summation order is not deterministic.
 *   F  device, real[3][M] (caller's marker order)   f  device, field[3][nz][ny][nx] */
int mls_spread(mls_ctx* ctx, const mls_transfer* T, const void* F, void* f, void* stream);

/* One direct-forcing transfer (text after Eq. 6, then Eq. 7): interpolate
 * U_l = sum_k phi_k^l u_k, form the IBM force F_l = (V_b,l - U_l) / dt that
 * drives the fluid velocity at marker l to the desired V_b,l, and spread
 * f_k += sum_l c_l phi_k^l F_l.  In single-precision contexts this is one
 * fused pass over the spreading tiles that reads phi once (a context whose
 * tile does not fit one block's shared memory composes the separate
 * kernels; double-precision contexts always do).
 *   u   device, field[3][nz][ny][nx]         Vb  device, real[3][M] desired velocity
 *   dt  time step (> 0)                      U   device, real[3][M] or NULL (not written)
 *   F   device, real[3][M] output forces     f   device, field[3][nz][ny][nx], accumulated
 * All marker arrays are in the caller's marker order.  Dropped markers get
 * U = 0 and F = 0 and add nothing to f.  The summation order of f is not
 * deterministic (as for mls_spread).
 * Errors: MLS_ERR_INVALID_ARG on NULL handles or arrays with M > 0, or
 * dt <= 0 or not finite. */
int mls_direct_forcing(mls_ctx* ctx, const mls_transfer* T, const void* u, const void* Vb, double dt,
                       void* U, void* F, void* f, void* stream);

/* mls_build_transfer followed by mls_direct_forcing of the same markers, in
 * one call (Section 2: Eqs. 3-6, then the direct-forcing transfer, text after
 * Eq. 6 and Eq. 7): the immersed-boundary step whose markers have just moved.
 * For MLS_EXACT with the linear basis the build kernel also interpolates U
 * and forms F_l = (V_b,l - U_l) / dt as each marker's shape functions are
 * formed (phi is not read back for the interpolation), and the spread of F
 * follows; other methods and bases run the two calls in turn.  Arguments,
 * outputs and errors are those of the two calls (U may be NULL); the results
 * equal theirs up to the rounding order of the sums.  Dropped markers get
 * U = 0 and F = 0 and add nothing to f. */
int mls_build_direct_forcing(mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M,
                             int32_t method, const void* u, const void* Vb, double dt, void* U, void* F, void* f,
                             void* stream);

/* Coarse-grained collision detection on the Eulerian mesh (Section 4): a
 * cell is a collision cell when markers of more than one body have it as
 * their home cell (the cell of the MLS support built by the last
 * mls_build_transfer on T).
 *   body        device, int32[M] body index of each marker (caller order);
 *               indices start at 1, markers with an index <= 0 take no part
 *   flag        device, int32[M] output (caller order): 1 when the marker's
 *               home cell is a collision cell, else 0 (also 0 for dropped
 *               markers)
 *   coll        device, int32[nz][ny][nx] or NULL: every cell holding
 *               participating markers gets the body index when they all
 *               belong to one body, -1 when they belong to several; other
 *               cells are not written (the caller zeroes the array, the
 *               method's initial state)
 *   n_colliding device, uint64 or NULL: incremented by the number of flagged
 *               markers
 * Errors: MLS_ERR_INVALID_ARG on NULL handles, or NULL body or flag with
 * M > 0. */
int mls_collisions(mls_ctx* ctx, const mls_transfer* T, const int32_t* body, int32_t* flag, int32_t* coll,
                   unsigned long long* n_colliding, void* stream);

/* Adaptive Lagrangian refinement of the forcing markers (Section 3, Fig. 5).
 * Each base triangle (V1, V2, V3) is split for the forcing step into
 *   level 0: itself; level 1: (V1, L1, V3), (L1, V2, V3) with L1 = (V1+V2)/2;
 *   level 2: (V1, V2, L2), (V2, V3, L2), (V3, V1, L2) with L2 the centroid;
 *   level 3: (V1, L31, L33), (L31, V2, L32), (L33, L32, V3), (L31, L32, L33)
 *            with L31, L32, L33 the midpoints of V1V2, V2V3, V3V1;
 * and every refined triangle gives one marker (centroid and area, as
 * mls_marker_prep).  The level is the smallest k <= max_level for which the
 * k+1 pieces have l^2 / (k+1) <= (ratio h)^2, where l^2 = 4 A / sqrt(3) is
 * the squared edge of the equilateral triangle of the same area A and h the
 * smallest width of the grid cell holding the base centroid (decided in
 * double precision); a centroid outside the grid keeps level 0.
 *   vertices device, real[n_vertices][3]   tri device, int32[n_tri][3]
 *   ratio    target l/h of the refined elements (> 0; 0.8 in the 0.7-0.9
 *            range the paper recommends)
 *   max_level 0..3
 *   x, area  device, real[3][capacity] and real[capacity] outputs (refined
 *            markers of triangle t are consecutive, triangles in order)
 *   parent   device, int32[capacity] output: base triangle of each marker
 *   level    device, int32[n_tri] output, or NULL
 *   n_markers host, int64 output: the number of refined markers
 * Synchronizes `stream` (the count is read back).  A triangle with an invalid
 * vertex index gives one NaN marker (as mls_marker_prep).
 * Errors: MLS_ERR_CAPACITY when n_markers > capacity (n_markers is still set
 * and the markers past capacity are not written); MLS_ERR_INVALID_ARG on NULL
 * pointers, negative sizes, ratio <= 0 or max_level outside 0..3. */
int mls_refine_markers(mls_ctx* ctx, const void* vertices, int64_t n_vertices, const int32_t* tri, int64_t n_tri,
                       double ratio, int32_t max_level, int64_t capacity, void* x, void* area, int32_t* parent,
                       int32_t* level, int64_t* n_markers, void* stream);

/* Borrowed device views of the last build (no synchronisation). */
int mls_transfer_view(const mls_transfer* T, mls_transfer_arrays* out);

/* Synchronise `stream`, then read the counters of the last build.  Returns
 * MLS_OK, or MLS_ERR_OUT_OF_DOMAIN when out->dropped > 0. */
int mls_transfer_status(const mls_transfer* T, void* stream, mls_status* out);

/* Fast-MLS table of the context (built on demand on `stream`):
 * real[n_classes][n_sub^3][MLS_TABLE_ROW], sub-node order
 * s = (s_z*n + s_y)*n + s_x, class = home index along the one non-uniform
 * axis (0 when all are uniform); a row holds the 27 exact shape-function
 * values of the sub-node (k = 9 c + 3 b + a) and one zero pad, so rows are
 * 16-byte aligned. */
#define MLS_TABLE_ROW 28
int mls_fast_table(mls_ctx* ctx, void* stream, const void** table, int64_t* n_classes, int32_t* n_sub);

/* Build without allocating.  The paper has no counterpart: this is a
 * convenience of the library for callers that cannot call cudaMalloc when
 * they build, for example a flow solver whose device memory all comes from
 * its own pool, or a time step in which a device allocation would
 * synchronise the whole device.  It computes exactly what
 * mls_build_transfer computes, with these differences:
 *   - the results go to caller-owned device buffers laid out like
 *     mls_transfer_arrays with capacity ld_phi (>= M):
 *       phi real[27][ld_phi], c real[ld_phi], home int32[ld_phi], perm int32[ld_phi];
 *   - the tile-sort workspace lives in one static device array of
 *     MLS_NOALLOC_SCRATCH_BYTES (about 5.3 MB) that every GPU which loads
 *     the library holds until the process exits;
 *   - limits: M <= MLS_NOALLOC_MAX_MARKERS and the context's spreading-tile
 *     count + 1 <= MLS_NOALLOC_MAX_BINS, else MLS_ERR_CAPACITY;
 *   - MLS_FAST needs the context's fast-MLS table to exist already (build it
 *     at set-up with mls_fast_table, which allocates), else MLS_ERR_UNSUPPORTED;
 *   - MLS_SURROGATE is not offered (its exact-MLS fallback and network
 *     buffers are not part of the static array): MLS_ERR_UNSUPPORTED;
 *   - no counters are returned: dropped markers are those with home = -1.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is kept for the life of the
 * process, which assumes the device's primary context lives as long: after
 * cudaDeviceReset the kept address is stale and the call must not be used.  All calls share the one array: calls that
 * overlap on the GPU (other streams, other contexts on the same device)
 * race and corrupt each other's results, so serialise them.  The context's
 * device must be current.  Calls no cudaMalloc or cudaFree. */
#define MLS_NOALLOC_MAX_MARKERS 262144
#define MLS_NOALLOC_MAX_BINS 266240
#define MLS_NOALLOC_SCRATCH_BYTES 5293312
int mls_build_transfer_noalloc(mls_ctx* ctx, const void* x, const void* area, int64_t M, int32_t method,
                               void* phi, void* c, int32_t* home, int32_t* perm, int64_t ld_phi, void* stream);

/* ---- learned surrogate (not in the paper) ------------------------------
 * On a grid uniform in all but one axis the shape functions of a marker depend
 * only on its offset t in the home cell and the width ratios along the
 * non-uniform axis (Section 2, the premise of fast-MLS).  A 6-64-64-27 network
 * (tanh hidden layers) maps the features
 *   t_x, t_y, t_z, ln(D_{i-1}/D_i), ln(D_{i+1}/D_i), ln(D_i/D_u)
 * (D: widths along the non-uniform axis, z when all are uniform; D_u: width of
 * the first other axis) to the 27 shape functions.  Its output is projected
 * orthogonally onto {sum phi = 1, sum phi xi = 0} (linear reproduction); a
 * marker whose residual then exceeds residual_max takes the exact-MLS value.
 * Parameters are float32, stored flat as W1[64][6], b1[64], W2[64][64],
 * b2[64], W3[27][64], b3[27] (MLS_MLP_PARAMS values); builds evaluate the
 * network with bfloat16 operands and float32 accumulation on tensor cores. */
#define MLS_MLP_PARAMS 6363

typedef struct {
  int64_t n_samples;     /* training set size, default 1048576 */
  int32_t epochs;        /* passes over the set, default 128 */
  int32_t batch;         /* minibatch size, 128..65536 and a multiple of 128, default 1024 */
  double lr;             /* initial Adam learning rate, default 3e-3 */
  double lr_final;       /* cosine-decayed final learning rate, default 1e-6 */
  uint64_t seed;         /* sample, minibatch and initialisation draws, default 1805011135 */
} mls_train_options;

int mls_train_options_default(mls_train_options* o);

/* Train the context's surrogate on the GPU (synchronous): draw n_samples
 * training points (offsets and, on a stretched grid, home cells of the
 * non-uniform axis) with the splitmix64 counter generator, label them with
 * exact-MLS shape functions computed in double, then run Adam on the mean
 * squared error with the library's forward/backward kernels.  `loss` (may be
 * NULL) receives the mean loss of the last epoch.  Allocates its workspace.
 * MLS_ERR_UNSUPPORTED for more than one non-uniform axis. */
int mls_surrogate_train(mls_ctx* ctx, const mls_train_options* o, void* stream, double* loss);

/* Copy the flat float32 parameters out of (set = 0) or into (set = 1) the
 * context; `host` holds MLS_MLP_PARAMS values.  Synchronous. */
int mls_surrogate_params(mls_ctx* ctx, float* host, int64_t n, int32_t set);

/* Training points first .. first+count-1 of a seed, as mls_surrogate_train
 * draws them: X device float[count][6], T device float[count][27]. */
int mls_surrogate_samples(mls_ctx* ctx, int64_t first, int64_t count, uint64_t seed, float* X, float* T,
                          void* stream);

/* Network on given inputs: X device float[B][6] -> Y device float[B][27].
 * mode MLS_F32: the float32 training path; MLS_BF16: the bfloat16 tensor-core
 * path builds use (before projection). */
int mls_surrogate_forward(mls_ctx* ctx, const float* X, int32_t B, int32_t mode, float* Y, void* stream);

/* Mean squared error over outputs and batch and its gradient for the current
 * parameters: X device float[B][6], T device float[B][27]; grad device
 * float[MLS_MLP_PARAMS]; loss device float[1].  B a multiple of 128. */
int mls_surrogate_loss_grad(mls_ctx* ctx, const float* X, const float* T, int32_t B, float* grad, float* loss,
                            void* stream);

/* ---- checkpoint / resume ------------------------------------------------
 * The context's marker-independent state: the fast-MLS table (Section 2,
 * Fig. 1b/1c; real[n_classes][n_sub^3][27] shape functions at the sub-Eulerian
 * points) when an MLS_FAST build or mls_fast_table has made it, and the
 * surrogate's float32 parameters when trained or set.  The file holds a
 * versioned header, a 64-bit key over the grid (n, periodic, every face), eps,
 * n_sub, the basis size and the real precision, the present blocks, and a
 * trailing checksum.
 *
 * mls_save: synchronises the device, writes `path` (host file name) through a
 * temporary "<path>.partial" that is renamed into place.  A context with
 * neither block writes a header-only file.  MLS_ERR_INVALID_ARG when the file
 * cannot be written; CUDA errors as MLS_ERR_CUDA.
 *
 * mls_load: reads and validates the whole file before changing the context;
 * then allocates the table if absent, copies it in (after a device
 * synchronise, so launches still using the old table finish first), and sets
 * the surrogate parameters as mls_surrogate_params(set = 1) does.  An
 * existing table is overwritten in place: its device address, and so any
 * CUDA graph captured with it, stays valid.
 * MLS_ERR_INVALID_ARG for a missing or unreadable file, a bad magic, version,
 * checksum or layout, or a key that differs from this context's (another grid
 * or option set), and MLS_ERR_UNSUPPORTED for surrogate parameters in a
 * context that cannot hold them; the context is then unchanged.  Only a CUDA
 * failure while copying (MLS_ERR_CUDA) can leave it partly loaded: a new
 * table without the file's surrogate parameters.  Both are synchronous. */
int mls_save(mls_ctx* ctx, const char* path);
int mls_load(mls_ctx* ctx, const char* path);

/* Per-kernel CUDA-event timing on the launching stream (off by default).
 * mls_timing_read synchronises the device, returns up to `max` accumulated
 * records in `out`, their count in `n`, and resets the accumulators. */
int mls_timing_enable(mls_ctx* ctx, int32_t on);
int mls_timing_read(mls_ctx* ctx, mls_kernel_time* out, int32_t max, int32_t* n);

const char* mls_strerror(int32_t code);
const char* mls_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MLS_GB300_H */
