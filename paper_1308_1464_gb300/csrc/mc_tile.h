// mc_tile.h -- tile geometry of the fused sweep, shared by host code (tensor
// maps, launch sizes) and the kernel.
#pragma once

namespace mc {

// Output columns of one warp band: 32 lanes own columns i0-1 .. i0+30;
// lanes 1..29 have both neighbours they need (limiter and transverse terms
// read lanes l-1 .. l+2), so 29 columns per band are written.
constexpr int BAND_W = 29;
constexpr int BAND_LANES = 32;

// elements per 16 bytes
__host__ __device__ constexpr int align_elems(int es) { return 16 / es; }
// TMA box width: 33 columns (i0-2 .. i0+30) plus room to round the start
// down to a 16-byte boundary, rounded up to 16 bytes
__host__ __device__ constexpr int box_w(int es)
{
    return ((33 + align_elems(es) - 1 + align_elems(es) - 1) / align_elems(es)) * align_elems(es);
}
// rows per TMA stage and stages in flight per warp
__host__ __device__ constexpr int stage_rows(int es) { return es == 4 ? 8 : 4; }
constexpr int NSTAGE = 3;
// bytes one TMA box delivers (the mbarrier transaction count) ...
__host__ __device__ constexpr int box_bytes(int es, int neq)
{
    return neq * stage_rows(es) * box_w(es) * es;
}
// ... and the stage pitch in shared memory (128-byte aligned destinations)
__host__ __device__ constexpr int stage_bytes(int es, int neq)
{
    return ((box_bytes(es, neq) + 127) / 128) * 128;
}
constexpr int SWEEP_WARPS = 4;
__host__ __device__ constexpr int sweep_smem_bytes(int es, int neq)
{
    return 128 + SWEEP_WARPS * NSTAGE * stage_bytes(es, neq);
}
// compile-time schemes of the fused step (see sweep_task)
constexpr int MODE_GENERAL = 0, MODE_TRANS2 = 1, MODE_FAST = 2;
constexpr int DEFAULT_TILE_ROWS = 64;
// state planes of any solver (Euler 4, variable-coefficient acoustics 5)
constexpr int BC_MAX_PLANES = 5;
// the default layout's long tasks: this many tiles of rows each (a task of r
// rows marches r + 3 rows, so longer ones re-read fewer halo rows)
constexpr int TALL_TILES = 2;
// attempts per captured graph of the time-step loop
constexpr int GRAPH_CHUNK = 50;

}  // namespace mc
