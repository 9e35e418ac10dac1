// Shared constants and launchers of the radius-query kernels.
#pragma once

#include "si_host.h"
#include "si_internal.cuh"
#include "si_walk.cuh"

namespace si {

constexpr int kQueryThreads = 128;   // per-query kernels
constexpr int kClassThreads = 256;   // per-query kernel with shared-memory class tables
constexpr int kInlineSort = 24;      // lists up to this length are sorted while written
constexpr int kDenseCap = 512;       // lists a warp of the dense path sorts in shared memory
constexpr int kCellThreads = 512;
constexpr int kCellCap = 2560;       // staged candidates per query cell
constexpr int kCellMaxQ = 512;       // queries of one cell in one block
constexpr int kCellTCap = 512;       // target cells of the cell-level sphere
constexpr int kSortWarps = 8;
constexpr int kSortWarpCap = 2048;   // lists a warp sorts in shared memory
constexpr int kSortBlockCap = 16384; // lists a block sorts in shared memory

size_t cell_smem_bytes();
si_status launch_cell_pass(const GridDev &g, const WalkParams &P, const Band &B, unsigned flags,
                           const int *heavy, int *big, int *work, int *over, long long *counts,
                           long long *cell_rec, int *scratch, long long scr_cap, unsigned long long *scr_top,
                           cudaStream_t st);
// Groups of heavy cells (si_group.cu): splits the heavy list into 2 x 2 x 2
// groups and the cells served one at a time (solo), and serves the groups.
size_t group_smem_bytes();
si_status launch_cell_group(const GridDev &g, const WalkParams &P, const Band &B, unsigned flags,
                            const int *heavy, int *groups, int *solo, int *work, int *big, int *over,
                            long long *counts, long long *cell_rec, int *scratch, long long scr_cap,
                            unsigned long long *scr_top, const unsigned long long *grow, int n_grow,
                            cudaStream_t st);
si_status launch_cell_expand(const GridDev &g, const int *heavy, const long long *cell_rec, const int *scratch,
                             int4 *items, int *blocks, const long long *offsets, int *ids, long long cap,
                             cudaStream_t st);

// Non-empty list method (si_list.cu): every (query, point) pair tested.
si_status launch_list(const GridDev &dv, const Band &B, unsigned flags, const int *list, int64_t m,
                      const float4 *ipos, long long *counts, const long long *off, int *ids, long long cap,
                      bool write, cudaStream_t st);
si_status gather_input(const si_grid *g, const GridDev &dv, float4 *ipos, cudaStream_t st);

}  // namespace si
