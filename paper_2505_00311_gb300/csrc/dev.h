// dev.h -- device views of a program (plain structs passed to the kernels by value),
// shared by the kernels and the host code that launches them.
#pragma once
#include "state.h"

namespace pdcs {

// Device view of one problem and its iterate state (passed by value).
// Rows of a CSR matrix binned by length for the SpMV (see spmv_binned).
constexpr int kSpmvMaxBins = 6;  // lane counts 32, 16, 8, 4, 2, 1
struct SpmvBins {
    int nbins;
    int blk[kSpmvMaxBins + 1];  // first block of each bin; blk[nbins] = grid size
    int row[kSpmvMaxBins + 1];  // first entry of each bin in the row list
    int lanes[kSpmvMaxBins];
};

// Sliced storage of a CSR matrix for the SpMV (see spmv_sliced): rows of at most
// kSliceMaxLen entries sorted by length (longest first) and cut into slices that one warp
// reads: a slice gives S lanes to each of its 32 / S rows (S = 2^slice_lg, chosen so that
// a lane takes at most kSlicePairsPerLane pairs of entries) and pads every row with
// columns -1 and values 0 to the slice's width W (a multiple of 2 S).  Pair p of slice
// row j sits at slice_off[s] + 64 q + 2 (j S + g) with p = q S + g: at step q the warp
// reads 64 consecutive entries.  Longer rows follow, each contiguous (long_rp), one warp
// per row.
constexpr int kSliceMaxLen = 512;
constexpr int kSlicePairsPerLane = 8;
struct SlicePlan {
    int nslices;
    int nlong;             // rows longer than kSliceMaxLen
    int nb_long;           // blocks of the long rows (first in the grid)
    int grid;              // nb_long + blocks of the slices
    const int* slice_off;  // nslices + 1 entry offsets (multiples of 64)
    const unsigned char* slice_lg;  // log2 of the lanes per row of each slice
    const int* out_row;    // 32 per slice: row j of the slice (j < 32 / S; -1 beyond or for padding)
    const int* long_row;   // nlong rows of A
    const int* long_rp;    // nlong + 1 entry offsets
};

// Rows of one SOC tile staged in shared memory (32 bytes each: the FP64 value, its weight
// and inverse weight, FP32 copies of the entry and of the weight), per warp
// (pdcs_options.soc_lane_entries > 0).
constexpr int kSocTileRows = 256;

// Grid-wise SOC cones (team.cuh): at least kTeamMinDim rows; a team takes at least
// kTeamMinRows x entries per block.  kTeamQ: quantities of one team sum.
constexpr int kTeamMinDim = 4096;
constexpr int kTeamMinRows = 512;
constexpr int kTeamQ = 4;

// Primal cone blocks (x2 in K_p): one block of pc_reduce / pc_apply per kPcChunk variables
// of a cone.
constexpr int kPcChunk = 1024;
enum PcMode { kPcHat = 0, kPcCand = 1, kPcLam = 2 };  // sources of pc_reduce / pc_apply

template <typename T>
struct Dev {
    int m, n;
    // scaled matrix K~ and its transpose, each stored bin by bin for the SpMV (row
    // pointer over the binned rows; binned row i is row listK[i] / listKT[i])
    const int* rp;
    const int* ci;
    const T* val;
    const int* rpT;
    const int* ciT;
    const T* valT;
    // scaled data
    const T* c;
    const T* h;
    const T* l;
    const T* u;
    const double* dr;
    const double* dc;
    // iterate state (xh and xh1: the two x-hat buffers, Ctrl::xsel picks the current one)
    T *x, *xh, *x0, *kty, *ktyh, *kty0, *xsum;
    T* xh1;
    int px_f0;  // first primal partial slot of the fused K' product's blocks (= primal_update's grid)
    T *y, *yh, *y0, *kx, *kxh0, *kxh1, *kx0, *ysum;
    // cone layout (internal row order): [0, m_zero) zero rows, [m_zero, m_scalar)
    // nonnegative rows, then SOC / RSOC blocks, then exp cones (3 rows each)
    int m_zero, m_scalar;
    int n_soc;
    const int* soc_off;
    const int* soc_dim;
    const unsigned char* soc_rot;
    float* soc_lam;        // last SOC root per cone (FP32 start of the next search)
    const double* soc_w;   // per SOC row: weight of the dual projection, (dr_row / dr_first)^2
    const double* soc_wp;  // per SOC row: weight of the primal projection, (dr_first / dr_row)^2
    int exp_row0, n_exp;
    const unsigned char* exp_kind;  // per exp-region block: 1 for K_exp^* (EXP_DUAL); null when none
    float* exp_L;          // last log-offset per exp cone
    const double* exp_lg;  // per exp cone: log dr of its three rows
    // SOC tiles of the FP64 dual update (see dual_soc_tiles): the cones sorted by dimension
    // (largest first), grouped in tiles of 32 / S cones of one lane-group size S, each tile
    // staged in shared memory; cones of more than kSocTileRows rows come last ("large",
    // a warp each on global memory)
    int n_tiles, n_large, nb_tiles;       // nb_tiles: blocks of the tiles (one tile per warp)
    const int* tile_cone0;                // n_tiles + 1: first cone of each tile in soc_order
    const int* tile_row0;                 // n_tiles + 1: first staged row of each tile in soc_trow
    const unsigned char* tile_lg;         // log2 S per tile
    const int* soc_order;                 // tiled cones, then the large ones
    const int* soc_so;                    // per tiled cone (as soc_order): its staged row offset in the tile
    const int* soc_trow;                  // internal row of each staged row, tile by tile
    // grid-wise projection of large SOC / RSOC cones (see team.cuh): entry e projects cone
    // team_cone[e] with blocks [team_b0[e], team_b0[e] + team_g[e]) of a cooperative launch
    // of team_nb blocks; soc_huge[c] = 1 for those cones, which the other SOC loops skip
    int team_nb, n_team;
    const int* team_cone;
    const int* team_b0;
    const int* team_g;
    unsigned* team_bar;              // [count, generation] per entry
    double* team_part;               // 2 * team_nb * kTeamQ partial slots
    const unsigned char* soc_huge;   // per cone, or null when no cone is projected by a team
    int team_gb0;                    // dual-update partial slot of team block 0
    int team_kb0;                    // primal-side KKT partial slot of team block 0
    // blocks of the cone-structured kernels: exp cones in [0, nb_exp), SOC cones in the
    // next nb_soc, scalar rows in the last nb_scal (the costliest work is dispatched first)
    int nb_scal, nb_soc, nb_exp;
    int exp_pb;  // exp cones per exp block (threads beyond it idle): spreads them over all SMs
    int nb_primal;
    // reductions and control
    double* part;
    PartLayout pl;
    Ctrl* ctrl;
    // check buffers (always FP64): candidates, their products, scratch
    double* xc;    // 2 n
    double* yc;    // 2 m
    double* kxc;   // 2 m
    double* ktyc;  // 2 n
    double* scr;   // 2 m scratch for projections of residuals
    // original-scale data for the unscaled KKT (FP64)
    const double* l_orig;
    const double* u_orig;
    // scaled data in FP64 for the checks (equal to c, h, l, u when T is double)
    const double* c64;
    const double* h64;
    const double* l64;
    const double* u64;
    // FP32 copies of the SOC weights and exp log-scales (FP32 iterates)
    const float* soc_w32;
    const float* exp_lg32;
    // learned starting point of the exp root search (kExpMlpParams floats), or null
    const float* exp_mlp;
    // primal cone blocks x2 in K_p (FP64 single programs): variables [pc_lo, pc_lo + pc_len)
    // in n_pc SOC / RSOC cones (first variable pc_off[k], size pc_dim[k], pc_rot[k] = 1 for
    // RSOC), pc_nch chunks of kPcChunk for the largest; scratch per source q (x-hat, or the
    // two candidates): pc_ss[(q n_pc + k) pc_nch + b] sums of squares, pc_t[q n_pc + k] first
    // entries, pc_mu[q pc_len + j - pc_lo] the projected reduced costs; pc_slot0: first
    // ||dx||^2 partial slot of pc_apply (n_pc pc_nch slots after primal_update's)
    int n_pc, pc_lo, pc_len, pc_nch, pc_slot0;
    const int* pc_off;
    const int* pc_dim;
    const unsigned char* pc_rot;
    double* pc_ss;
    double* pc_t;
    double* pc_mu;
    // SpMV plans of K and K': bins and the row each binned row stands for
    SpmvBins binsK, binsKT;
    const int* listK;
    const int* listKT;
};

}  // namespace pdcs
