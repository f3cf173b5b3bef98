// mc_halo.cu -- ghost layers of one block of a decomposed grid.
//
// A grid split into blocks (one per device or rank) steps each block on its
// own; before every step the two ghost layers along a side shared with
// another block are that block's two interior layers next to the side, and
// sides on the global boundary keep their boundary kind (LeVeque 2002, §7.1
// and §21.8: the update of a cell reads cells up to two away, diagonal
// neighbours included through the transverse terms).  The fill runs in two
// phases so that corner ghosts come out as in the single-grid fill: x ghosts
// of the interior rows first, then y ghosts across the full padded width
// (the x ghost columns included).  This file holds the kernels of those
// phases: packing a side's two interior layers into a dense strip,
// unpacking a received strip into the ghost layers, and the directional
// fill of the sides whose kind is a physical boundary.  It also holds the
// repacking of a whole interior between the dense [meqn][my][mx] order and
// the padded layout, which lets a host transfer of a state move one
// contiguous block.
#include "mc_internal.h"
#include "mc_tile.h"

namespace mc {

namespace {

struct HaloArgs {
    int mx, my, meqn;
    long long ld_x, ld_field, x_offset;
};

__host__ __device__ inline long long halo_count(const HaloArgs& a, int side)
{
    return side < 2 ? (long long)a.meqn * a.my * 2 : (long long)a.meqn * 2 * (a.mx + 4);
}

// element offset of the cell of strip position t: interior cells next to
// the side (pack) or the ghost cells on the side (unpack)
__device__ inline long long halo_cell(const HaloArgs& a, int side, bool ghost, long long t)
{
    int m, i, j;
    if (side < 2) {                      // [meqn][my][2], columns in increasing i
        const long long per = 2LL * a.my;
        m = int(t / per);
        const int r = int(t % per);
        j = r >> 1;
        const int c = r & 1;
        i = side == 0 ? (ghost ? c - 2 : c) : (ghost ? a.mx + c : a.mx - 2 + c);
    } else {                             // [meqn][2][mx + 4], rows in increasing j
        const long long W = a.mx + 4;
        const long long per = 2 * W;
        m = int(t / per);
        const int r = int(t % per);
        const int k = int(r / W);
        i = int(r % W) - 2;
        j = side == 2 ? (ghost ? k - 2 : k) : (ghost ? a.my + k : a.my - 2 + k);
    }
    return (long long)m * a.ld_field + (long long)(j + 2) * a.ld_x + a.x_offset + i;
}

// The state is qa, or qb when cur is given and *cur == 1 (the buffer index a
// block's device-side time-step loop keeps).
template <typename T>
__global__ void halo_pack_kernel(const T* qa, const T* qb, const int* cur, T* __restrict__ buf,
                                 const HaloArgs a, int side)
{
    const T* __restrict__ q = (cur && *cur) ? qb : qa;
    const long long n = halo_count(a, side);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        buf[t] = q[halo_cell(a, side, false, t)];
}

template <typename T>
__global__ void halo_unpack_kernel(const T* __restrict__ buf, T* qa, T* qb, const int* cur,
                                   const HaloArgs a, int side)
{
    T* __restrict__ q = (cur && *cur) ? qb : qa;
    const long long n = halo_count(a, side);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        q[halo_cell(a, side, true, t)] = buf[t];
}

// source index of ghost index g (g < 0 or g >= n) by the boundary kinds of
// the low and high sides; a reflecting wall (mirror about the boundary)
// flips the normal component.  Repeats while the image is still outside,
// which only happens for n < 2.
__device__ inline int ghost_source(int g, int n, int lo_kind, int hi_kind, bool& flip)
{
    for (int it = 0; it < 4 && (g < 0 || g >= n); it++) {
        const int kind = g < 0 ? lo_kind : hi_kind;
        if (kind == MC_BC_PERIODIC) {
            g = ((g % n) + n) % n;
        } else if (kind == MC_BC_EXTRAP) {
            g = g < 0 ? 0 : n - 1;
        } else {
            g = g < 0 ? -g - 1 : 2 * n - 1 - g;
            flip = !flip;
        }
    }
    return g < 0 ? 0 : (g >= n ? n - 1 : g);
}

template <typename T>
struct DirArgs {
    T* qa;
    T* qb;
    const int* cur;                       // fill qa (cur == 0 or null) or qb (cur == 1)
    HaloArgs h;
    int bc[4];
};

// dir 0: x ghost columns of the interior rows; dir 1: y ghost rows across
// the full padded width.  Sides of kind MC_BC_GIVEN are left as they are.
template <typename T>
__global__ void bc_dir_kernel(const DirArgs<T> a, int dir)
{
    const HaloArgs& h = a.h;
    T* q = (a.cur && *a.cur) ? a.qb : a.qa;
    const long long W = h.mx + 4;
    const long long n = dir == 0 ? 4LL * h.my : 4LL * W;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        int i, j, si, sj, side;
        bool flip = false;
        if (dir == 0) {
            j = int(t >> 2);
            const int g = int(t & 3);
            i = g < 2 ? g - 2 : h.mx + g - 2;
            side = g < 2 ? 0 : 1;
            if (a.bc[side] == MC_BC_GIVEN) continue;
            si = ghost_source(i, h.mx, a.bc[0], a.bc[1], flip);
            sj = j;
        } else {
            const int g = int(t / W);
            i = int(t % W) - 2;
            j = g < 2 ? g - 2 : h.my + g - 2;
            side = g < 2 ? 2 : 3;
            if (a.bc[side] == MC_BC_GIVEN) continue;
            sj = ghost_source(j, h.my, a.bc[2], a.bc[3], flip);
            si = i;
        }
        const long long dst = (long long)(j + 2) * h.ld_x + h.x_offset + i;
        const long long src = (long long)(sj + 2) * h.ld_x + h.x_offset + si;
        const int fm = dir == 0 ? 1 : 2;  // normal momentum of the side
        // all planes' loads first, so their latencies overlap (a ghost's
        // source is never a ghost this phase writes)
        T v[BC_MAX_PLANES];
#pragma unroll
        for (int m = 0; m < BC_MAX_PLANES; m++)
            if (m < h.meqn) v[m] = q[m * h.ld_field + src];
#pragma unroll
        for (int m = 0; m < BC_MAX_PLANES; m++)
            if (m < h.meqn) q[m * h.ld_field + dst] = (flip && m == fm) ? -v[m] : v[m];
    }
}

HaloArgs halo_args(const mc_problem& p, const mc_layout& lay)
{
    return HaloArgs{p.mx, p.my, (int)lay.meqn, lay.ld_x, lay.ld_field, lay.x_offset};
}

int grid_for(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    return b < 1 ? 1 : int(b);
}

}  // namespace

long long halo_elems(const mc_problem& p, int side)
{
    const HaloArgs a{p.mx, p.my, solver_meqn(p.solver), 0, 0, 0};
    return halo_count(a, side);
}

cudaError_t halo_launch_cur(const mc_problem& p, const mc_layout& lay, void* qa, void* qb,
                            const int* cur_dev, void* buf, int side, bool pack, cudaStream_t s)
{
    const HaloArgs a = halo_args(p, lay);
    const int blocks = grid_for(halo_count(a, side));
    if (p.dtype == MC_F64) {
        if (pack) halo_pack_kernel<double><<<blocks, 256, 0, s>>>(
            static_cast<const double*>(qa), static_cast<const double*>(qb), cur_dev,
            static_cast<double*>(buf), a, side);
        else halo_unpack_kernel<double><<<blocks, 256, 0, s>>>(
            static_cast<const double*>(buf), static_cast<double*>(qa), static_cast<double*>(qb),
            cur_dev, a, side);
    } else {
        if (pack) halo_pack_kernel<float><<<blocks, 256, 0, s>>>(
            static_cast<const float*>(qa), static_cast<const float*>(qb), cur_dev,
            static_cast<float*>(buf), a, side);
        else halo_unpack_kernel<float><<<blocks, 256, 0, s>>>(
            static_cast<const float*>(buf), static_cast<float*>(qa), static_cast<float*>(qb),
            cur_dev, a, side);
    }
    return cudaGetLastError();
}

cudaError_t halo_launch(const mc_problem& p, const mc_layout& lay, const void* src, void* dst,
                        int side, bool pack, cudaStream_t s)
{
    void* q = const_cast<void*>(pack ? src : static_cast<const void*>(dst));
    void* buf = pack ? dst : const_cast<void*>(src);
    return halo_launch_cur(p, lay, q, q, nullptr, buf, side, pack, s);
}

namespace {

// One interior row (m, j) per loop step: dense row m * my + j holds
// row_words words, the layout row starts at word lay_base(m, j).  Word W is
// 16 bytes when every row start is 16-byte aligned on both sides, else one
// element.
template <typename W>
__global__ void dense_repack_kernel(const W* __restrict__ src, W* __restrict__ dst, int my,
                                    int rows, long long row_words, long long ld_x_w,
                                    long long ld_field_w, long long x_offset_w, bool to_layout)
{
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int m = r / my, j = r - m * my;
        const long long dense0 = (long long)r * row_words;
        const long long lay0 = (long long)m * ld_field_w + (long long)(j + 2) * ld_x_w + x_offset_w;
        const W* s = src + (to_layout ? dense0 : lay0);
        W* d = dst + (to_layout ? lay0 : dense0);
        for (long long i = threadIdx.x; i < row_words; i += blockDim.x) d[i] = s[i];
    }
}

template <typename W>
cudaError_t repack_as(const void* src, void* dst, int my, int rows, long long row_words,
                      long long ld_x_w, long long ld_field_w, long long x_offset_w, bool to_layout,
                      int sms, cudaStream_t s)
{
    const int blocks = rows < 8 * sms ? rows : 8 * sms;
    dense_repack_kernel<W><<<blocks, 256, 0, s>>>(static_cast<const W*>(src), static_cast<W*>(dst), my,
                                                 rows, row_words, ld_x_w, ld_field_w, x_offset_w,
                                                 to_layout);
    return cudaGetLastError();
}

}  // namespace

cudaError_t dense_repack_launch(const mc_problem& p, const mc_layout& lay, const void* src,
                                void* dst, bool to_layout, int sms, cudaStream_t s)
{
    const long long es = lay.elem_bytes;
    const int rows = lay.meqn * p.my;
    const uintptr_t a = reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst);
    // 16-byte words when the row length, both bases and every layout row
    // start are multiples of 16 bytes
    const bool v16 = (p.mx * es) % 16 == 0 && a % 16 == 0 && (lay.ld_x * es) % 16 == 0 &&
                     (lay.ld_field * es) % 16 == 0 && ((lay.x_offset + 2 * lay.ld_x) * es) % 16 == 0;
    if (v16) {
        const long long k = 16 / es;
        return repack_as<uint4>(src, dst, p.my, rows, p.mx / k, lay.ld_x / k, lay.ld_field / k,
                                lay.x_offset / k, to_layout, sms, s);
    }
    if (es == 8)
        return repack_as<unsigned long long>(src, dst, p.my, rows, p.mx, lay.ld_x, lay.ld_field,
                                             lay.x_offset, to_layout, sms, s);
    return repack_as<unsigned int>(src, dst, p.my, rows, p.mx, lay.ld_x, lay.ld_field, lay.x_offset,
                                   to_layout, sms, s);
}

cudaError_t bc_dir_launch(const mc_problem& p, const mc_layout& lay, void* qa, void* qb,
                          const int* cur_dev, int dir, cudaStream_t s)
{
    const HaloArgs h = halo_args(p, lay);
    const long long n = dir == 0 ? 4LL * p.my : 4LL * (p.mx + 4);
    const int blocks = grid_for(n);
    if (p.dtype == MC_F64) {
        DirArgs<double> a{static_cast<double*>(qa), static_cast<double*>(qb), cur_dev, h,
                          {p.bc[0], p.bc[1], p.bc[2], p.bc[3]}};
        bc_dir_kernel<double><<<blocks, 256, 0, s>>>(a, dir);
    } else {
        DirArgs<float> a{static_cast<float*>(qa), static_cast<float*>(qb), cur_dev, h,
                         {p.bc[0], p.bc[1], p.bc[2], p.bc[3]}};
        bc_dir_kernel<float><<<blocks, 256, 0, s>>>(a, dir);
    }
    return cudaGetLastError();
}

}  // namespace mc
