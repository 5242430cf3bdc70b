// Internal structures shared by the translation units of libftlm.
#pragma once

#include <stdint.h>

#include <array>
#include <atomic>
#include <string>
#include <vector>

#include "ftlm.h"

namespace ftlm {

constexpr int kMaxG = 128;      // group order supported on the GPU path (4 elements per lane)
constexpr int kMaxGHost = 512;  // group order supported by the host group module
constexpr int kMaxD = 12;       // irrep dimension supported on the GPU path (Section 3's limit)
constexpr int kMaxBonds = 64;   // bonds per cluster on the GPU path
constexpr int kMaxB = 32;       // right-hand sides per H·v launch
constexpr int kPMaxK = 10;      // blocks per packed set (compile-time shapes)
constexpr int kMaxSteps = 512;  // Lanczos steps per chain

// Record of one representative in a packed set: label, first row of its
// segment in the packed vector, stabilizer subgroup id.
struct alignas(16) HvRec {
    uint64_t label;
    uint32_t off;
    uint32_t sid;
};

// Entry of the optional per-sector table of ladder flips (the paper's two-phase
// design, Section 3): the flipped state's representative (index in the
// sector), the minimising element g*, the bond and the sign of the flip
// (bit 7: s_i^- s_j^+), and the representative's stabilizer id.  A
// representative's entries follow the H·v kernel's flip order.
struct alignas(8) HvEntry {
    uint32_t tgt;
    uint8_t g;
    uint8_t esign;
    uint16_t sid;
};
static_assert(sizeof(HvEntry) == 8, "entry tables are read as 8-byte words (two per 16-byte load)");

// Packed set: K blocks of one sector whose rows are interleaved by
// representative, in lifted coordinates: representative r owns the W = sum_k
// d_k rows (k, gamma), gamma < d_k, holding V_k(r) x_k(r) (Eq. 11's V_r maps a
// block's n_k(r) coefficients of r isometrically into the irrep space).  K = 1
// is a single block.  Built by packed.cu.
struct PackedSet {
    int K = 0;
    int W = 0;          // sum of d_k: rows of a representative with trivial stabilizer
    int shape = -1;     // compiled shape id (see packed.cu), -1 if none matches
    int dims[kPMaxK] = {};
    uint64_t rows = 0;  // packed rows = n_reps * W
    HvRec *d_rec = nullptr;         // [n_reps]: label, off = index * W, stabilizer id
    uint8_t *d_ntab = nullptr;      // [n_sid][K] n_k(sid)
    uint8_t *d_wtab = nullptr;      // [n_sid] sum_k n_k(sid)
    double *d_P[kPMaxK] = {};       // block k: [n_sid][d_k][d_k] projector V V^T
    float *d_Pf[kPMaxK] = {};
    double *d_rhoT = nullptr;       // concatenated padded rho(g)^T tables
    float *d_rhoTf = nullptr;
    int rho_total = 0, rho_totalf = 0;
    int rho_off[kPMaxK] = {}, rho_offf[kPMaxK] = {};
    std::vector<uint8_t> h_wtab;
    uint32_t neg = 0;  // spin-flip sectors: bit k set when block k is a Gamma- block
    size_t device_bytes = 0;
};

ftlm_status fail(ftlm_status st, const char *fmt, ...);
void clear_error();
void count_launch(int n = 1);
bool profiling_on();
unsigned long long *profile_flip_counter();

// A real-irreducible representation: an irrep of real Frobenius-Schur type
// (fs = 1), the real form of a complex pair Gamma + conj(Gamma) (fs = 0,
// dimension 2 d_Gamma) or of a quaternionic irrep (fs = -1, dimension
// 2 d_Gamma).  kappa = <chi, chi> = 1, 2, 4 is the dimension of its real
// commutant; a single-partner-row block counts each level kappa times, so its
// weight in Eqs. 5 and 14 is dim / kappa.
struct Irrep {
    int dim = 0;
    int fs = 1;                 // Frobenius-Schur indicator of the complex constituent
    std::vector<double> chars;  // [G], trace of rho
    std::vector<double> rho;    // [G][dim][dim] real orthogonal
    int kappa() const { return fs == 1 ? 1 : (fs == 0 ? 2 : 4); }
    int weight() const { return dim / kappa(); }
};

struct GroupData {
    int N = 0;
    int G = 0;
    std::vector<int32_t> perms;  // [G][N], canonical order, perms[g*N + k] = pi_g(k)
    std::vector<int32_t> inv;    // [G]
    std::vector<int32_t> mult;   // [G][G], mult[g*G + h] = index of g h
    std::vector<int32_t> bonds;  // [n_bonds][2]
    double J = 1.0;
    std::vector<Irrep> irreps;
    int n_bonds() const { return (int)bonds.size() / 2; }
};

// host group module (group.cpp)
ftlm_status build_group(int n_sites, int n_gens, const int32_t *gens, int n_bonds, const int32_t *bonds, double J,
                        GroupData &out);
ftlm_status compute_irreps(GroupData &g);
ftlm_status canonicalise_and_verify_irreps(GroupData &g, std::vector<Irrep> &irreps, double tol);

}  // namespace ftlm

struct ftlm_group {
    ftlm::GroupData d;
};

// Packed-label sector on the device (basis.cu).
struct ftlm_sector {
    std::atomic<int> refs{1};
    // the group acting on the sector: G, or G x Z_2 with the spin flip at M = 0 (flip = 1), whose
    // element g + z |G| is stored as the signed permutation pi_g(k) + z N and whose irreps are
    // Gamma_i+ (2i) and Gamma_i- (2i + 1); G below is |G| of the site permutations alone
    ftlm::GroupData grp;
    int two_s = 0, two_M = 0, bits = 0, N = 0, G = 0, A = 0;
    int flip = 0;
    uint64_t flipc = 0;  // spin flip of a packed label: n ^ flipc (s = 1/2) or flipc - n (fields 2s - a_k)
    bool half = false;   // s = 1/2 with N <= 32: 32-bit labels, XOR flips
    uint64_t n_reps = 0, sector_dim = 0;
    uint64_t *d_labels = nullptr;   // [n_reps] ascending packed labels
    uint16_t *d_stab_id = nullptr;  // [n_reps] stabilizer subgroup id (0 = trivial)
    std::vector<std::array<uint64_t, 4>> stab_masks;  // per id: bit g of the group acting on the sector
    std::vector<std::vector<int>> stab_elems;         // per id
    uint32_t *d_bucket = nullptr;                     // [n_buckets + 1] first rep index of each bucket
    uint64_t *d_eoff = nullptr;                       // entry table (optional): [n_reps + 1] first entry
    ftlm::HvEntry *d_ent = nullptr;                   // [n_entries] per representative, in flip order
    uint64_t n_entries = 0;
    size_t entry_bytes = 0;
    int bucket_shift = 0;
    uint64_t n_buckets = 0;
    // H·v search tables
    uint32_t *d_lut = nullptr;   // s = 1/2: [nchunk][16][kMaxG] image of a 4-site nibble under g
    int n_chunks = 0;
    uint32_t *d_lut2 = nullptr;  // s = 1/2: [nchunk2][4][kMaxG] image of a 2-site chunk under g
    int n_chunks2 = 0;
    uint8_t *d_pos = nullptr;    // general s: [kMaxG][64] bit position of site k's field after g
    void *d_dtab = nullptr;      // [n_bonds][kMaxG] u32 XOR masks (s = 1/2) or int64 deltas (general)
    uint8_t *d_bonds = nullptr;  // [n_bonds][2] site pairs
    int *d_err = nullptr;        // device error word
    size_t device_bytes = 0;
};

struct ftlm_basis {
    ftlm_sector *sec = nullptr;
    int irrep = 0, d = 0;
    uint64_t dim = 0;
    uint64_t *d_off = nullptr;      // [n_reps + 1]
    // per stabilizer id: n_Gamma, sqrt|Stab|, V [d][d] (V[beta*d + k])
    uint8_t *d_ntab = nullptr;
    double *d_sqrtS = nullptr;
    float *d_sqrtSf = nullptr;
    double *d_V = nullptr;
    float *d_Vf = nullptr;
    // rho(g)^T per element with padded rows, [G][d][rho_row(d)]: rhoT[g][b][c] = rho(g)[c][b]
    double *d_rhoT = nullptr;
    float *d_rhoTf = nullptr;
    int rho_elems = 0, rho_elemsf = 0;  // padded table sizes (FP64, FP32)
    std::vector<uint8_t> h_ntab;
    ftlm::PackedSet *ps = nullptr;  // the block as a one-block packed set
    size_t device_bytes = 0;
};

// Several irrep blocks of one sector sharing one H·v launch (basis.cu, hv_multi_*.cu).
struct ftlm_multiblock {
    ftlm_sector *sec = nullptr;
    int K = 0;
    std::vector<ftlm_basis *> blocks;  // owned
    uint64_t *d_offm = nullptr;        // [n_reps][K] row offsets, interleaved
    uint8_t *d_ntab = nullptr;         // [K][n_sid]
    double *d_rhoT = nullptr;          // blocks' padded rho(g)^T tables concatenated
    float *d_rhoTf = nullptr;
    int rho_total = 0, rho_totalf = 0;
    std::vector<int> d, rho_off, rho_offf;
    ftlm::PackedSet *ps = nullptr;  // packed layout of the whole set (null if its shape is not compiled)
    size_t device_bytes = 0;
};

namespace ftlm {
void sector_release(ftlm_sector *s);
// packed.cu
ftlm_status packed_set_build(ftlm_sector *s, int K, const ftlm_basis *const *blocks, void *stream, PackedSet **out);
void packed_set_free(PackedSet *ps);
int packed_shape_id(int K, const int *dims);
}
