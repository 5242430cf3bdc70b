/*
 * ftlm.h — C ABI of the GB300 symmetry-adapted FTLM library.
 *
 * The library evaluates the matrix-free Hamiltonian action H·v of the
 * isotropic spin-s Heisenberg model (Eq. 1 of arXiv 2607.17429) in the basis
 * adapted to one S^z sector M and one real irrep Gamma of a site-permutation
 * group G (Sections 2.3-2.4, Eqs. 8-16), and runs the finite-temperature
 * Lanczos method on top of it (Section 2.2, Eqs. 4-7 and 14).
 *
 * Conventions used by every entry point:
 *  - Group elements are site permutations, gens[g*n_sites + k] = pi_g(k): the
 *    digit of site k moves to site pi_g(k) (Section 2.3), U(g)U(h) = U(gh).
 *    Elements are kept in canonical order: lexicographic order of the arrays
 *    (pi_g(0), ..., pi_g(N-1)); the identity is element 0.
 *  - Irreps are real orthogonal (Frobenius-Schur indicator +1, Section 3),
 *    ordered by dimension, then by character vector (canonical element order,
 *    rounded to 1e-8) descending; irrep 0 is the trivial irrep.
 *  - Spin and magnetisation are passed doubled: two_s = 2s, two_M = 2M.
 *  - Product states are stored packed, ceil(log2(2s+1)) bits per site with
 *    site k in the k-th bit field; this preserves the order of the paper's
 *    base-(2s+1) labels (Eq. 2), so orbit representatives (smallest label of
 *    the orbit, Section 2.3) are the same states.
 *  - Block vectors are row-major [dim][B]: row (r, k) of the block (k-th
 *    basis vector of representative r, Eq. 12 at partner row 1), B right-hand
 *    sides contiguous per row.  Rows follow the representatives in ascending
 *    label order, k = 0..n_Gamma(r)-1 (Eq. 13).
 *  - The caller owns every pointer it passes; the library owns opaque handles
 *    until the matching *_free.  Device pointers must stay valid until the
 *    work queued on the caller's stream has finished.
 *  - Every call returns an ftlm_status; on failure ftlm_last_error() gives a
 *    message (thread-local).  No call aborts, exits or traps on the device.
 *  - cuda_stream is a cudaStream_t (NULL = the legacy default stream).
 */
#ifndef FTLM_H
#define FTLM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FTLM_OK = 0,
    FTLM_EINVAL = 1,       /* bad argument (null pointer, out-of-range index or size) */
    FTLM_ENOTGROUP = 2,    /* generators are not permutations or close to a group above the size limit */
    FTLM_EBONDS = 3,       /* the bond list is not invariant under every group element (Section 3) */
    FTLM_EIRREP = 4,       /* irrep construction or verification failed (Section 3) */
    FTLM_EUNSUPPORTED = 5, /* d_Gamma > 5, complex/quaternionic irrep, |G| > 128 on the GPU path, labels > 64 bits */
    FTLM_ENOMEM = 6,       /* device or host allocation failed */
    FTLM_ECUDA = 7,        /* a CUDA runtime call failed */
    FTLM_ETIMEOUT = 8,     /* a bounded device-side wait gave up */
    FTLM_EINTERNAL = 9     /* a device bounds check tripped (e.g. a representative missing from the table) */
} ftlm_status;

/* Vector storage and H·v arithmetic.  FTLM_F16: FP16 storage of the packed
 * Lanczos vectors with FP32 arithmetic and FP64 reductions (Section 3's
 * half-precision storage mode, with the per-block power-of-two scale of
 * Section 4.2); offered by the packed entry points (ftlm_hv_packed and the
 * Lanczos calls). */
typedef enum { FTLM_F64 = 0, FTLM_F32 = 1, FTLM_F16 = 2 } ftlm_dtype;
typedef enum { FTLM_GAUSS = 0, FTLM_RADEMACHER = 1 } ftlm_rng;

typedef struct ftlm_group ftlm_group;   /* host: permutations, multiplication table, irreps, bonds */
typedef struct ftlm_sector ftlm_sector; /* device: representatives, stabilizers, lookup index of one (s, M) */
typedef struct ftlm_basis ftlm_basis;   /* device: one (s, M, Gamma) block on top of a sector */
typedef struct ftlm_multiblock ftlm_multiblock; /* device: several blocks of one sector, one H·v launch */

/* ---------------------------------------------------------------- group (host) */

/*
 * Close site-permutation generators into the group and compute its real irreps
 * (Section 3: closure, irreps from the regular representation, real form,
 * verification of unitarity, character orthogonality and sum d^2 = |G|).
 *   n_sites        number of sites N (1..64)
 *   gens           [n_gens][n_sites] host, gens[g][k] = pi_g(k)
 *   bonds          [n_bonds][2] host, site pairs of Eq. 1 (i != j)
 *   J              exchange constant of Eq. 1
 *   out            receives the new handle
 * Errors: FTLM_EINVAL, FTLM_ENOTGROUP (not permutations, or |G| > 512),
 *         FTLM_EBONDS (Section 3's bond-invariance check), FTLM_EIRREP.
 * Irreps are real-irreducible representations with real orthogonal matrices:
 * an irrep of real Frobenius-Schur type (fs = 1); for a pair Gamma, conj(Gamma)
 * of complex type (fs = 0) one entry, the real form of dimension 2 d_Gamma; for
 * a quaternionic irrep (fs = -1) its real form of dimension 2 d_Gamma.  A block
 * of a real form holds every level kappa = 2 (complex) or 4 (quaternionic)
 * times, so it enters Eqs. 5, 6 and 14 with the weight dim / kappa
 * (ftlm_group_weights) instead of d_Gamma.  Section 3 keeps a complex-arithmetic
 * path for those irreps instead; the real form computes the same thermal sums in
 * real arithmetic with the same vector length (2 D real numbers for D complex).
 */
ftlm_status ftlm_group_init(int n_sites, int n_gens, const int32_t *gens, int n_bonds, const int32_t *bonds,
                            double J, ftlm_group **out);

/*
 * Built-in clusters (Section 3's providers), built from coordinates with
 * nearest-neighbour bonds and J = 1: "icosahedron", "dodecahedron",
 * "icosidodecahedron" (I_h, 120), "cuboctahedron" (O_h, 48), "tetrahedron"
 * (T_d, 24), "dimer", "ring:N" (D_N), "square:LXxLY[:c4v|c2v|t]" (periodic
 * square lattice with its point group and translations, or translations only).
 */
ftlm_status ftlm_group_builtin(const char *name, ftlm_group **out);

/*
 * Group facts.  Any output pointer may be NULL.
 *   dims, fs: [n_irreps] (real dimension, Frobenius-Schur indicator);
 *   chars: [n_irreps][order] (traces of the real matrices, canonical element order).
 */
ftlm_status ftlm_group_info(const ftlm_group *g, int *n_sites, int *order, int *n_irreps, int *dims, int *fs,
                            double *chars);
/*
 * Weight of every irrep's block in Eqs. 5, 6 and 14 (the ftlm_block d_gamma):
 * dims / kappa with kappa = 1, 2, 4 for fs = 1, 0, -1.  weights: [n_irreps] host.
 */
ftlm_status ftlm_group_weights(const ftlm_group *g, int *weights);

/*
 * Export one irrep and the element table.  rho: [order][d][d] host,
 * rho[g][a][b] = rho_Gamma(g)_{ab} (NULL to skip).  perms: [order][n_sites]
 * (NULL to skip).
 * bonds: [n_bonds][2] (NULL to skip), n_bonds/J may be NULL.
 */
ftlm_status ftlm_group_irrep(const ftlm_group *g, int irrep, double *rho, int32_t *perms);
ftlm_status ftlm_group_bonds(const ftlm_group *g, int *n_bonds, int32_t *bonds, double *J);

/*
 * Replace the computed irreps by tabulated ones (Section 2.3: irrep matrices
 * "from standard tables or computed numerically").  rho_all holds, irrep after
 * irrep, [order][dims[i]][dims[i]] real matrices in canonical element order.
 * Every irrep must be a homomorphism with orthogonal matrices; its type comes
 * from <chi, chi> = 1, 2, 4 (real, complex pair, quaternionic); the characters
 * must be orthogonal with those norms and sum d^2 / kappa = |G| (Section 3's
 * checks, 1e-9); otherwise FTLM_EIRREP and the group is unchanged.  The irreps are re-sorted into the
 * canonical irrep order.  Sectors and blocks built before the call are unaffected.
 */
ftlm_status ftlm_group_set_irreps(ftlm_group *g, int n_irreps, const int *dims, const double *rho_all);

void ftlm_group_free(ftlm_group *g);

/* ---------------------------------------------------------------- basis (device) */

/*
 * Irrep-independent preparation of one S^z sector (Section 3's first phase):
 * enumerate the sector on the GPU (digit sum N s + M, Section 2.1), keep the
 * orbit representatives (smallest label, Section 2.3) in ascending order, their
 * stabilizers (Eq. 8) and a bucket index for label lookup.  Queued on
 * cuda_stream; the call synchronises that stream before returning.
 * The sector keeps a copy of the group; the group may be freed afterwards.
 * Errors: FTLM_EINVAL (M out of range, N s + M not an integer),
 *         FTLM_EUNSUPPORTED (N * bits > 64, |G| > 128, more than 2^32 - 1
 *         representatives), FTLM_ENOMEM, FTLM_ECUDA.
 */
ftlm_status ftlm_build_sector(const ftlm_group *g, int two_s, int two_M, void *cuda_stream, ftlm_sector **out);
/*
 * The M = 0 sector under G x Z_2, Z_2 the global spin flip m -> -m (Section
 * 2.2: at M = 0 the flip commutes with H and with the site permutations, and
 * each irrep Gamma splits into Gamma+ and Gamma-, roughly halving the blocks).
 * Element (g, z) has index g + z|G|; representatives are orbit minima under
 * both; the flip image of a label is arithmetic (digits 2s - a_k), so the
 * search adds no permutation.  The sector's irreps are Gamma_i+ at index 2i
 * (rho(g, z) = rho_i(g)) and Gamma_i- at 2i + 1 (rho(g, z) = (-1)^z rho_i(g)),
 * the canonical order of G x Z_2; blocks, packed sets, H·v, Lanczos and
 * entry tables take these indices.  Errors as ftlm_build_sector, and
 * FTLM_EINVAL when N s is not an integer (no M = 0 sector).
 */
ftlm_status ftlm_build_sector_flip(const ftlm_group *g, int two_s, void *cuda_stream, ftlm_sector **out);
ftlm_status ftlm_sector_info(const ftlm_sector *s, uint64_t *n_reps, uint64_t *sector_dim, size_t *device_bytes);
/* The group acting on the sector: its order (|G|, or 2|G| with the spin flip), its irrep count and the flag. */
ftlm_status ftlm_sector_symmetry(const ftlm_sector *s, int *order, int *n_irreps, int *flip);
/* labels: [n_reps] packed labels; stab_mask: [n_reps][W] bit g of the mask set when element g fixes r,
 * W = 2 words (128-bit masks) for a plain sector, 4 (256 bits, index g + z|G|) with the spin flip. */
ftlm_status ftlm_sector_export(const ftlm_sector *s, uint64_t *labels, uint64_t *stab_mask);
void ftlm_sector_free(ftlm_sector *s);

/*
 * Entry table of a sector (Section 3: the two-phase design, where a
 * preparation pass maps every ladder flip of every representative to its
 * target representative and group element, and each H·v then reads the
 * table instead of searching).  ftlm_sector_build_entries runs that pass once
 * (the representative search and lookup of Eq. 15 for every flip of Eq. 3)
 * and keeps the table on the device with the sector: 8 bytes per flip plus 8
 * per representative, counted in ftlm_sector_info's device_bytes; n_entries
 * (may be NULL) receives the flip count.  From then on every packed H·v and
 * Lanczos call on blocks of this sector reads the table (the same flips in
 * the same order as the search, so the results are bitwise those of the
 * search path; a single block at one right-hand side runs one thread per
 * representative and sums its flips in entry order, equal to the search path
 * to rounding).  Synchronises cuda_stream; FTLM_ENOMEM if the table does not
 * fit.  ftlm_sector_free_entries drops the table (back to the search).
 * Neither may run while another call uses the sector.
 */
ftlm_status ftlm_sector_build_entries(const ftlm_sector *s, void *cuda_stream, uint64_t *n_entries);
ftlm_status ftlm_sector_free_entries(const ftlm_sector *s);

/*
 * Irrep-dependent preparation (Section 3's second phase): per stabilizer
 * subgroup n_Gamma (Section 2.3), V_r (Eq. 11: modified Gram-Schmidt over the
 * columns of (1/|Stab|) sum_h rho(h) in column order, residual threshold 1e-8,
 * count checked against the character formula) and sqrt|Stab|; per
 * representative the row offset (prefix sum of n_Gamma, Eq. 13).
 * The block keeps the sector alive (reference counted).
 * Errors: FTLM_EINVAL (irrep index), FTLM_EUNSUPPORTED (dimension above 12,
 * Section 3's limit), FTLM_EIRREP, FTLM_ENOMEM, FTLM_ECUDA.
 */
ftlm_status ftlm_build_block(const ftlm_sector *s, int irrep, void *cuda_stream, ftlm_basis **out);

/* ftlm_build_sector followed by ftlm_build_block; the basis owns its sector. */
ftlm_status ftlm_build_basis(const ftlm_group *g, int two_s, int two_M, int irrep, void *cuda_stream,
                             ftlm_basis **out);
ftlm_status ftlm_basis_info(const ftlm_basis *b, uint64_t *n_reps, uint64_t *dim, size_t *device_bytes);
/*
 * Host copies for bit-exact tests (NULL = skip): labels [n_reps] packed,
 * stab_mask [n_reps][W] (W as in ftlm_sector_export), n_gamma [n_reps], offsets [n_reps + 1].
 */
ftlm_status ftlm_basis_export(const ftlm_basis *b, uint64_t *labels, uint64_t *stab_mask, uint8_t *n_gamma,
                              uint64_t *offsets);
void ftlm_basis_free(ftlm_basis *b);

/* ---------------------------------------------------------------- H·v (device) */

/*
 * y = H x in the (M, Gamma) block, B right-hand sides (1 <= B <= 32), one
 * launch on cuda_stream, asynchronous.  Per representative r (Eqs. 15-16 in
 * their Hermitian-transposed pull form):
 *   y[r,k] = J sum_<ij> m_i m_j x[r,k]
 *          + sum_{bond, sign} c_a sqrt(|Stab r'|/|Stab r|) [V_r^T rho(g_e) V_r' x_r']_k
 * where a is the flipped state (Eq. 3 gives c_a), r' = min O(a) and
 * a = U(g_e) r' are found by the in-kernel representative search, and r' is
 * looked up in the sorted representative table.
 *   x, y  device [dim][B] of double (FTLM_F64) or float (FTLM_F32), not aliased.
 * The call lifts x into the block's one-block packed layout, runs the packed
 * kernel (see ftlm_hv_packed) and lowers the result into y, with scratch from
 * the stream-ordered allocator (cudaMallocAsync) on cuda_stream.
 * Errors: FTLM_EINVAL (null pointers, B out of range), FTLM_ECUDA (launch).
 * A representative missing from the table (impossible for a consistent basis)
 * sets a device flag reported as FTLM_EINTERNAL by ftlm_basis_check; a
 * bounded wait that gave up is reported there as FTLM_ETIMEOUT.
 */
ftlm_status ftlm_hv(const ftlm_basis *b, ftlm_dtype dtype, int B, const void *x, void *y, void *cuda_stream);

/*
 * Synchronise cuda_stream and report (then clear) the device error word of the
 * basis's sector: FTLM_ETIMEOUT if a bounded wait gave up, FTLM_EINTERNAL if a
 * bounds check tripped, FTLM_OK otherwise.
 */
ftlm_status ftlm_basis_check(const ftlm_basis *b, void *cuda_stream);

/*
 * Several irrep blocks of one sector prepared for a shared H·v launch.  The
 * representative search and lookup of a flipped state are irrep independent
 * (Section 3 builds that part once per sector), so ftlm_hv_multi runs them
 * once per representative and then applies Eq. 15's contraction for every
 * block.  irreps: [n_blocks] indices (1 <= n_blocks <= 16); every block must
 * have dim < 2^32.  The set owns its blocks and keeps the sector alive.
 */
ftlm_status ftlm_build_multiblock(const ftlm_sector *s, int n_blocks, const int *irreps, void *cuda_stream,
                                  ftlm_multiblock **out);
ftlm_status ftlm_multiblock_info(const ftlm_multiblock *mb, int *n_blocks, uint64_t *dims, size_t *device_bytes);
/* Borrowed handle of block k (valid while the set lives), e.g. for ftlm_basis_export or ftlm_hv. */
ftlm_status ftlm_multiblock_block(const ftlm_multiblock *mb, int k, const ftlm_basis **out);
void ftlm_multiblock_free(ftlm_multiblock *mb);

/*
 * y_k = H x_k for every block k of the set in one launch (same result as
 * ftlm_hv per block).  x, y: host arrays of n_blocks device pointers, block k's
 * vectors [dim_k][B] of the chosen dtype.  Asynchronous on cuda_stream.
 */
ftlm_status ftlm_hv_multi(const ftlm_multiblock *mb, ftlm_dtype dtype, int B, const void *const *x, void *const *y,
                          void *cuda_stream);

/*
 * Packed layout of a multi-block set: the rows of every block of the set are
 * interleaved by representative, in lifted coordinates.  Representative i
 * (ascending label order) owns the W = sum_k d_k rows i W + Z_k + gamma
 * (Z_k = d_0 + ... + d_{k-1}, gamma < d_k) holding x~_k(r) = V_k(r) x_k(r):
 * the n_k(r) coefficients of r in block k (Eq. 13's rows of r) mapped into the
 * d_k-dimensional irrep space by the orthonormal columns of V_r (Eq. 11).  The
 * map is an isometry, so inner products and norms equal those of the block
 * vectors; for a trivial stabilizer V_r = I.  Vectors are [rows][B] with rows =
 * n_reps * W.  One flipped state's representative r' then owns one fixed-size
 * segment holding every block's coefficients, so one lookup and one gather
 * serve all blocks of Eq. 15.  Available for the compiled block shapes: a
 * single block of dimension 1..12, and the full real irrep sets of I_h, O_h and
 * T_d in canonical irrep order (every set built by ftlm_build_multiblock over
 * those irreps); rows below 2^32.
 *   ftlm_multiblock_packed_rows: *rows = n_reps * W (FTLM_EUNSUPPORTED if the
 *     set has no packed layout).
 *   ftlm_multiblock_pack: lift per-block vectors (host array of n_blocks device
 *     pointers, [dim_k][B] each) into one packed device vector [rows][B];
 *   ftlm_multiblock_unpack: the inverse, x_k(r) = V_k(r)^T x~_k(r).  Both
 *     synchronise cuda_stream.
 */
ftlm_status ftlm_multiblock_packed_rows(const ftlm_multiblock *mb, uint64_t *rows);
ftlm_status ftlm_multiblock_pack(const ftlm_multiblock *mb, ftlm_dtype dtype, int B, const void *const *blocks,
                                 void *packed, void *cuda_stream);
ftlm_status ftlm_multiblock_unpack(const ftlm_multiblock *mb, ftlm_dtype dtype, int B, const void *packed,
                                   void *const *blocks, void *cuda_stream);

/*
 * y = H x for every block of the set at once on packed vectors (Eqs. 15-16, the
 * same arithmetic as ftlm_hv per block, in lifted coordinates):
 *   y~_k(r) = P_k(r) z_k(r) / sqrt|Stab r| + diag(r) x~_k(r),
 *   z_k(r)  = sum_{bond, sign} c_a sqrt|Stab r'| rho_k(g_e) x~_k(r'),
 * with P_k(r) = V_k(r) V_k(r)^T.  One warp per representative searches and
 * looks up every flipped state once, gathers r''s whole segment (bulk copies
 * into shared memory when B * element size is a multiple of 16 bytes and x is
 * 16-byte aligned, lane loads otherwise) and contracts it with every block's
 * rho(g*)^T.  x, y: device [rows][B], not aliased, 1 <= B <= 32.  Asynchronous
 * on cuda_stream.  Errors: FTLM_EINVAL, FTLM_EUNSUPPORTED (no packed layout),
 * FTLM_ECUDA.  Device-side failures (a representative missing from the table,
 * a bounded wait that gave up) are reported by ftlm_basis_check on any block of
 * the set.
 */
ftlm_status ftlm_hv_packed(const ftlm_multiblock *mb, ftlm_dtype dtype, int B, const void *x, void *y,
                           void *cuda_stream);

/*
 * Autotuner of the packed H·v (no counterpart in the paper, which picks its
 * batch width from free memory).  With on = 1, the first packed H·v plan of
 * every (block shape, |G| class, label width, element type, B, gather path,
 * log2 of the representative count) key times the candidate geometries on that
 * plan's own vectors and keeps the fastest for the rest of the process: warps
 * per CTA, staging buffers in flight, rho tables in shared memory or read
 * through L1 (FP32), the own-row prefetch, representatives per tile.  Every
 * candidate computes identical rows; only timing changes (Lanczos alpha/beta
 * can change at the rounding level through the reduction tiling).  on = 0
 * turns tuning off (the built-in choice, cached results kept); on = -1 also
 * clears the cache.  ftlm_autotune_report writes one text line per cached key
 * (choice, its time and the default's) into buf (len bytes, NUL-terminated).
 */
ftlm_status ftlm_set_autotune(int on);
ftlm_status ftlm_autotune_report(char *buf, size_t len);

/*
 * Cycle budget of every bounded device-side wait of the H·v kernels (the
 * mbarrier waits for bulk copies); 0 restores the default of 2^32 cycles
 * (about two seconds).  A wait that runs out records FTLM_ETIMEOUT, which
 * ftlm_basis_check (and the Lanczos calls) return; the warp then waits, with
 * the default budget, for its copies already in flight before it stops.
 * Library-wide; meant for tests of the timeout path.
 */
ftlm_status ftlm_set_wait_limit(uint64_t cycles);

/*
 * Test and benchmark inputs at any block size (no counterpart in the paper).
 * ftlm_fill_label_keyed writes the label-keyed block vector x [dim][B] (device,
 * dtype, 1 <= B <= 64): the entry of row k of representative r and right-hand
 * side b is, with L the base-(2s+1) label of r (Eq. 2) and SplitMix64 as
 * published by Steele, Lea and Flood (OOPSLA'14), all arithmetic mod 2^64,
 *   z = L * 4096 + k * 64 + b + seed * 0x632BE59BD9B4E019,
 *   x = (splitmix64(z) >> 11) * 2^-52 - 1  (in [-1, 1), rounded to the dtype).
 * Any row can be regenerated from its label alone.  Asynchronous on cuda_stream.
 * ftlm_basis_rows looks up n packed labels (host array): first_row[i] = the
 * block row of representative labels[i] (-1 if it is not a representative) and
 * n_rows[i] = its n_Gamma (host outputs).  Synchronises cuda_stream.
 */
ftlm_status ftlm_fill_label_keyed(const ftlm_basis *b, ftlm_dtype dtype, int B, uint64_t seed, void *x,
                                  void *cuda_stream);
ftlm_status ftlm_basis_rows(const ftlm_basis *b, int n, const uint64_t *labels, int64_t *first_row, int *n_rows,
                            void *cuda_stream);

/* ---------------------------------------------------------------- Lanczos / FTLM */

/*
 * R independent Lanczos chains on the block (Section 2.2), batched through one
 * H·v launch per step (at most 32 chains per batch).  Start vectors:
 * Philox4x32-10 with key (low 32 bits of seed, low 32 bits of block_id) and
 * counter (row low, row high, chain, 0); Gaussian by Box-Muller on two 53-bit
 * uniforms, or Rademacher +-1 from bit 0; each chain normalised in FP64.
 * Recurrence: w = H v_j; alpha_j = <v_j, w>; w -= alpha_j v_j + beta_j v_{j-1};
 * beta_{j+1} = |w|; v_{j+1} = w / beta_{j+1}, run on the block's packed
 * (lifted) vectors with the normalisation folded into scale factors: the
 * stored vector is u_j = v_j / s_j and alpha_j = s_j^2 <u_j, H u_j>.  Dot
 * products and norms use exact products of the stored values (FP32 vectors in
 * FTLM_F32), double-float sums per representative and lane, FP64 beyond; the
 * order is fixed, so repeated runs give identical coefficients.  The N_L-step
 * loop is captured in a CUDA graph (FTLM_NO_GRAPH=1 launches it directly).
 * A chain stops after step j when beta_{j+1} <= tol (|alpha_j| + beta_j)
 * (tol = 1e-12 for FP64, 1e-6 for FP32) or when j + 1 = min(n_steps, dim).
 *   alpha, beta   host [R][n_steps]; beta[r][j] = beta_{j+1} (beta[r][m-1] is
 *                 the final residual norm); entries past steps_done are 0.
 *   steps_done    host [R].
 * Device work memory (3 packed [rows][B] vectors and reduction scratch) is
 * allocated and freed by the call.  Synchronises cuda_stream before returning.
 * FTLM_ETIMEOUT / FTLM_EINTERNAL report device-side failures of the H·v.
 */
ftlm_status ftlm_lanczos(const ftlm_basis *b, ftlm_dtype dtype, int R, int n_steps, uint64_t seed,
                         uint64_t block_id, ftlm_rng rng, void *cuda_stream, double *alpha, double *beta,
                         int *steps_done);

/*
 * ftlm_lanczos on every block of a multi-block set in lockstep.  Sets with a
 * packed layout run the packed path of ftlm_lanczos_sets (one H·v launch and
 * one update launch per step for all blocks, captured in a CUDA graph);
 * others take one ftlm_hv_multi launch plus per-block recurrence kernels per
 * step.  Block k
 * draws its start vectors with block_ids[k]; results equal ftlm_lanczos per
 * block up to rounding.  alpha, beta: host [n_blocks][R][n_steps];
 * steps_done: host [n_blocks][R].
 */
ftlm_status ftlm_lanczos_multi(const ftlm_multiblock *mb, ftlm_dtype dtype, int R, int n_steps, uint64_t seed,
                               const uint64_t *block_ids, ftlm_rng rng, void *cuda_stream, double *alpha,
                               double *beta, int *steps_done);

/*
 * ftlm_lanczos_multi on several packed sets at once, for instance every S^z
 * sector of a cluster (Section 2.2's block-factorised FTLM): all sets must
 * come from the same group (same permutations, bonds, J and irreps), the same
 * spin and the same irreps in the same order, and have a packed layout.  Each
 * kernel of a step is one launch over the representatives of every set (the
 * sets are the parts of a persistent tile walk), and the step loop is one
 * CUDA graph.  block_ids: host [n_sets][K]; alpha, beta: host
 * [n_sets][K][R][n_steps]; steps_done: host [n_sets][K][R].
 */
ftlm_status ftlm_lanczos_sets(int n_sets, const ftlm_multiblock *const *sets, ftlm_dtype dtype, int R, int n_steps,
                              uint64_t seed, const uint64_t *block_ids, ftlm_rng rng, void *cuda_stream,
                              double *alpha, double *beta, int *steps_done);

/*
 * Ritz values and weights of tridiagonal matrices on the GPU in FP64 (implicit
 * QL with Wilkinson shifts, first eigenvector row only; Section 2.2).
 *   n_chains, m[c] = steps of chain c, alpha/beta host [n_chains][ld];
 *   theta, w: host [n_chains][ld] (entries past m[c] set to 0).
 */
ftlm_status ftlm_ritz(int n_chains, int ld, const int *m, const double *alpha, const double *beta, double *theta,
                      double *w, void *cuda_stream);

typedef struct {
    int two_M;              /* 2M of the block's sector */
    int d_gamma;            /* the irrep's weight (Eq. 14): ftlm_group_weights */
    uint64_t dim;           /* block dimension D_{M,Gamma} (Eq. 13) */
    int R;                  /* number of chains */
    int ld;                 /* leading dimension of alpha/beta (>= max steps) */
    const int *steps_done;  /* [R] */
    const double *alpha;    /* [R][ld] */
    const double *beta;     /* [R][ld] */
} ftlm_block;

/*
 * FTLM thermal sums over all blocks on the GPU in FP64 (Eqs. 5-7 with the
 * weight mult_M d_Gamma D/R of Eq. 14; mult_M = 2 for M > 0, 1 for M = 0;
 * k_B = mu_B = 1).  Ritz pairs from ftlm_ritz's method; exponentials shifted
 * by the global minimum Ritz value E0.  C = beta^2 <(H - <H>)^2> (centred),
 * chi = g^2 beta sum mult_M M^2 Z_M / sum mult_M Z_M.
 *   T: host [n_T] (> 0); outputs lnZ, E, C, chi host [n_T] (any may be NULL),
 *   E0 host [1] (may be NULL).  Synchronises cuda_stream.
 */
ftlm_status ftlm_thermo(int n_blocks, const ftlm_block *blocks, int n_T, const double *T, double g, double *lnZ,
                        double *E, double *C, double *chi, double *E0, void *cuda_stream);

/*
 * Same thermal sums as ftlm_thermo, for callers that cannot allocate device
 * memory: code running inside a process whose device memory is entirely
 * reserved by another allocator or pool (a serving runtime, a framework's
 * caching allocator), or code that must not trigger the device-wide
 * synchronisation that cudaMalloc/cudaFree can cause.  The paper has no
 * counterpart; this is an interface variant of ftlm_thermo.
 *
 * Every pointer is a DEVICE pointer owned by the caller, chain-major:
 *   m [n_chains] steps per chain (0 <= m <= ld), alpha/beta [n_chains][ld]
 *   (beta[c][j] couples steps j and j+1), weight [n_chains] = mult_M d_Gamma
 *   D_{M,Gamma} / R of the chain's block (Eq. 14), msq [n_chains] = M^2 of
 *   that block, T [n_T] > 0; outputs out [4][n_T] = lnZ, E, C, chi and E0 [1].
 * The intermediate Ritz pairs live in a fixed file-scope device array of
 * 2 x 2^19 doubles (8 MiB, held by every GPU that loads the library until the
 * process exits); n_chains * ld above 2^19 (or ld above 512) is rejected with
 * FTLM_EINVAL before any GPU work.  The call allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.  The array itself is reserved by the
 * CUDA driver when it loads the library's device code on a device: at library
 * load with CUDA_MODULE_LOADING=EAGER, otherwise (CUDA's default, lazy
 * loading) at the first use of that code on the device, which may be this
 * call.  A call with n_chains = 0 (every other argument ignored) only makes
 * the array and the call's kernels resident on the current device and returns
 * FTLM_OK: make it before handing the rest of the device memory to a pool.
 * The array's address is looked up on every call (valid after a context
 * reset).  All calls share the one array and it keeps the last call's
 * contents; calls that overlap on the GPU (other
 * streams, other host threads) race on it and must be serialised by the
 * caller.  Synchronises cuda_stream before returning; FTLM_EINTERNAL if a
 * chain's steps exceed ld or the eigensolve does not converge.
 */
ftlm_status ftlm_thermo_noalloc(int n_chains, int ld, const int *m, const double *alpha, const double *beta,
                                const double *weight, const double *msq, int n_T, const double *T, double g,
                                double *out, double *E0, void *cuda_stream);

/* ---------------------------------------------------------------- serving loop */

/*
 * Serving loop for many independent FTLM jobs on one GPU.  The paper has no
 * counterpart beyond choosing its batch width from free memory (Section 3);
 * this is the continuous-batching form of ftlm_lanczos.
 *
 * A job is one block (2M, irrep) of a group's cluster at spin 2s with R
 * chains (1..32) of n_steps (1..512) Lanczos steps, its own block_id (Philox
 * key word 1 of the start vectors) and the seed, generator and dtype of
 * ftlm_lanczos.  The server owns a scheduler thread and n_workers worker
 * threads, each with its own CUDA stream on the device current at creation.
 *  - Admission: jobs are admitted in submission order while the device bytes
 *    charged stay within cap_bytes.  Charged are the resident sector tables
 *    (one per group, 2s, 2M; shared by every job on them), the resident
 *    block tables (one per sector and irrep) and each admitted job's Lanczos
 *    vectors and state (3 packed vectors of rows x min(R, 32) elements plus a
 *    few MB).  A sector is estimated from its dimension before it is built and
 *    charged its actual size after.  Tables that no admitted job references
 *    are evicted least recently used first when room is needed.  A job that
 *    does not fit even with nothing else admitted fails with FTLM_ENOMEM; a
 *    job that would fit later waits (head of line).
 *  - Waves: an idle worker takes the oldest admitted job and every admitted
 *    job with the same group, 2s, irrep, R, dtype, rng and seed (up to
 *    max_parts), and runs them as the parts of one packed Lanczos launch
 *    (ftlm_lanczos_sets' machinery, S^z sectors may differ); each part stops
 *    at its own n_steps.  A job's coefficients equal those of ftlm_lanczos on
 *    the same block, seed and block_id up to rounding.
 * The group must stay valid until every job submitted on it has finished.
 * ftlm_server_submit validates the job and returns its id at once
 * (FTLM_EINVAL for bad arguments).  ftlm_server_wait blocks until the job has
 * finished (timeout_s < 0: no limit; FTLM_ETIMEOUT if it runs out, the job
 * keeps running), fills info and the host arrays alpha/beta [R][n_steps] and
 * steps_done [R] (any may be NULL), returns the job's status and forgets the
 * job.  Times in info are seconds since the server was created.
 * ftlm_server_free stops the threads after the waves in flight; jobs not yet
 * started are dropped.
 */
typedef struct ftlm_server ftlm_server;
typedef struct {
    const ftlm_group *group;
    int two_s, two_M, irrep;
    int R, n_steps;
    uint64_t seed, block_id;
    ftlm_rng rng;
    ftlm_dtype dtype;
} ftlm_job;
typedef struct {
    ftlm_status status;
    int d_gamma;            /* the irrep's weight (ftlm_group_weights) */
    uint64_t dim;
    double t_submit, t_admit, t_start, t_done;
} ftlm_job_info;
typedef struct {
    uint64_t submitted, completed, failed, waves, parts;
    uint64_t sectors_built, sector_hits, blocks_built, block_hits, evictions;
    size_t cap, charged, peak_charged, resident_table_bytes;
    int queued, ready, running_waves;
} ftlm_server_stats;

ftlm_status ftlm_server_create(size_t cap_bytes, int n_workers, int max_parts, ftlm_server **out);
ftlm_status ftlm_server_submit(ftlm_server *srv, const ftlm_job *job, uint64_t *job_id);
ftlm_status ftlm_server_wait(ftlm_server *srv, uint64_t job_id, double timeout_s, ftlm_job_info *info,
                             double *alpha, double *beta, int *steps_done);
ftlm_status ftlm_server_stats_get(ftlm_server *srv, ftlm_server_stats *out);
void ftlm_server_free(ftlm_server *srv);

/* ---------------------------------------------------------------- profiling */

/*
 * Library-wide counters (tracing support; no counterpart in the paper beyond
 * its wall times).  kernel_launches counts every kernel the library launched
 * since the last reset.  While profiling is enabled, every H·v launch is
 * bracketed by CUDA events on its stream (events recorded inside the Lanczos
 * graph for its launches); hv_ms is their summed device time, hv_rows the
 * summed rows * B, and hv_flips the ladder flips (Eq. 3 terms) the packed
 * H·v processed, counted on the device.  ftlm_profile_get waits for the
 * device.
 */
typedef struct {
    uint64_t kernel_launches;
    uint64_t hv_launches;
    double hv_ms;
    uint64_t hv_rows;
    uint64_t hv_flips;
} ftlm_profile;
ftlm_status ftlm_profile_enable(int on);
ftlm_status ftlm_profile_reset(void);
ftlm_status ftlm_profile_get(ftlm_profile *out);

/*
 * Roofline denominators measured on the current device (no counterpart in the
 * paper; it reports hardware counters only).  Each probe runs a fixed grid of
 * 4 CTAs per SM, once to warm up and once timed with CUDA events on
 * cuda_stream, and writes the sustained rate to *rate:
 *   FTLM_PEAK_LOP3 / _MIN_U32 / _ADD_U64  integer lane-operations per second
 *   FTLM_PEAK_FFMA32 / _DFMA64            fused multiply-adds per second (lanes)
 *   FTLM_PEAK_LDS32                       conflict-free 32-bit shared loads per second
 *   FTLM_PEAK_GATHER                      bytes per second of random aligned segments
 *                                         of seg bytes (a multiple of 16) read from a
 *                                         device buffer of span bytes (the segments
 *                                         drawn from the first 2^floor(log2(span/seg)));
 *                                         segments of at most 64 bytes one per lane,
 *                                         longer ones one per warp
 *   FTLM_PEAK_STREAM                      bytes per second (read + write) of a copy
 *                                         of span bytes
 * span and seg are ignored by the arithmetic probes.  The gather and stream
 * probes allocate their buffers (span <= 64 GiB) and free them before
 * returning.  Synchronises cuda_stream.
 */
enum {
    FTLM_PEAK_LOP3 = 0,
    FTLM_PEAK_MIN_U32 = 1,
    FTLM_PEAK_ADD_U64 = 2,
    FTLM_PEAK_FFMA32 = 3,
    FTLM_PEAK_DFMA64 = 4,
    FTLM_PEAK_LDS32 = 5,
    FTLM_PEAK_GATHER = 6,
    FTLM_PEAK_STREAM = 7
};
ftlm_status ftlm_peak_probe(int kind, uint64_t span, int seg, void *cuda_stream, double *rate);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *ftlm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FTLM_H */
