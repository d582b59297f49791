// vkt_bricks.cu -- BrickDecompose (Sec. 3.2, "domain decomposition algorithms": a volume is
// split into subgrids, optionally with ghost cells for interpolation).
//
// Brick (kx, ky, kz) covers the source voxels [o, o + s) with o = (kx bx, ky by, kz bz) and
// s = min(b, dims - o) per axis, and is stored as a volume of s + 2 g voxels per axis whose
// voxel (i, j, k) is the source voxel clamp(o - g + (i, j, k)): ghost cells inside the volume
// copy the neighbouring bricks' voxels, ghost cells beyond a face repeat the face voxel (the
// clamp-to-edge rule of ApplyFilter).  One launch copies every brick.  Bricks with ghost
// cells on a source a tensor map describes take brick planes as the unit (k_bricks_planes:
// one TMA box per plane, one funnel shift per output word); otherwise a CTA takes a run of
// brick rows: with a 16-byte aligned source and 4-byte aligned bricks (every torch
// allocation) the rows are staged in shared memory by asynchronous 16-byte copies and
// written as blocks or words (k_bricks_staged), else a warp copies four rows at a time, its
// lanes consecutive x (k_bricks).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>

#include "vkt_internal.h"
#include "vkt_tile.cuh"

namespace vkt {
namespace {

constexpr int NT = 256;
constexpr int NWARP = NT / 32;
constexpr int MIN_ROWS_PER_CTA = 64;

struct BrickDesc {
    void* dst;
    int ox, oy, oz;      // source origin of the brick's interior
    int dx, dy, dz;      // stored dims (interior + 2 ghost)
};

// The bricks' storage pointers travel as a kernel parameter (no per-call table upload);
// a launch takes up to MAXB bricks (blockIdx.y), the rest of a brick's description follows
// from its index in the brick grid.
constexpr int MAXB = 3968;   // 31.7 KB of pointers, within the 32 KB parameter limit
struct BrickPtrs {
    void* p[MAXB];
};
struct BrickGrid {
    int nx, ny, nz;          // volume
    int bx, by, bz;          // brick size
    int cx, cy;              // bricks along x and y
    int first;               // index of the launch's first brick
    int ghost;
};

__device__ __forceinline__ BrickDesc brick_at(const BrickPtrs& P, const BrickGrid& G)
{
    const int i = G.first + static_cast<int>(blockIdx.y);
    const int kx = i % G.cx, ky = (i / G.cx) % G.cy, kz = i / (G.cx * G.cy);
    BrickDesc d;
    d.dst = P.p[blockIdx.y];
    d.ox = kx * G.bx;
    d.oy = ky * G.by;
    d.oz = kz * G.bz;
    d.dx = min(G.bx, G.nx - d.ox) + 2 * G.ghost;
    d.dy = min(G.by, G.ny - d.oy) + 2 * G.ghost;
    d.dz = min(G.bz, G.nz - d.oz) + 2 * G.ghost;
    return d;
}

bool valid_volume(const vktStructuredVolume_impl* v) { return v && v->magic == VKT_VOLUME_MAGIC; }

int elem_bytes(vktDataFormat f) { return f == vktDataFormatUint8 ? 1 : (f == vktDataFormatUint16 ? 2 : 4); }

__device__ __forceinline__ int clampd(int v, int lo, int hi) { return min(max(v, lo), hi); }

// T: the voxel's storage type as an unsigned integer of its size (bit-exact copies).  A warp
// copies RP brick rows at a time, its lanes consecutive x; a lane issues its RP x EPL loads
// before its stores (brick rows are short, so the reads in flight come from several rows).
constexpr int RP = 4, EPL = 3;

template <typename T>
__global__ void __launch_bounds__(NT)
    k_bricks(const T* __restrict__ src, const BrickPtrs P, const BrickGrid G, int rows_per_cta)
{
    const int nx = G.nx, ny = G.ny, nz = G.nz, ghost = G.ghost;
    const BrickDesc b = brick_at(P, G);
    const int rows = b.dy * b.dz;
    const int r0 = blockIdx.x * rows_per_cta;
    if (r0 >= rows) return;
    const int r1 = min(rows, r0 + rows_per_cta);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* dst = static_cast<T*>(b.dst);
    // dst columns [0, left) repeat source column 0, [right, dx) column nx-1; in between
    // they are one contiguous span of the source row (plain indexing, no clamps)
    const int sx0 = b.ox - ghost;
    const int left = clampd(-sx0, 0, b.dx);
    const int right = clampd(nx - sx0, left, b.dx);
    const int n = right - left;
    for (int rb = r0 + warp * RP; rb < r1; rb += (NT / 32) * RP) {
        const T* s[RP];
        T* d[RP];
#pragma unroll
        for (int q = 0; q < RP; ++q) {
            const int r = min(rb + q, r1 - 1);
            const int k = r / b.dy, j = r - k * b.dy;
            const int sz = clampd(b.oz - ghost + k, 0, nz - 1);
            const int sy = clampd(b.oy - ghost + j, 0, ny - 1);
            const T* srow = src + (static_cast<int64_t>(sz) * ny + sy) * nx;
            T* drow = dst + static_cast<int64_t>(r) * b.dx;
            if (rb + q < r1) {
                for (int i = lane; i < left; i += 32) drow[i] = __ldg(srow);
                for (int i = right + lane; i < b.dx; i += 32) drow[i] = __ldg(srow + nx - 1);
            }
            s[q] = srow + sx0 + left;
            d[q] = drow + left;
        }
        const int nq = min(RP, r1 - rb);
        for (int c0 = lane; c0 < n; c0 += 32 * EPL) {
            T v[RP][EPL];
#pragma unroll
            for (int q = 0; q < RP; ++q)
#pragma unroll
                for (int e = 0; e < EPL; ++e)
                    if (c0 + 32 * e < n) v[q][e] = __ldg(s[q] + c0 + 32 * e);
#pragma unroll
            for (int q = 0; q < RP; ++q) {
                if (q >= nq) break;
#pragma unroll
                for (int e = 0; e < EPL; ++e)
                    if (c0 + 32 * e < n) d[q][c0 + 32 * e] = v[q][e];
            }
        }
    }
}

// Staged variant (16-byte aligned source, 4-byte aligned bricks).  Byte-wide loads keep too
// few bytes in flight for short brick rows, so a CTA stages a batch of brick rows in shared
// memory first: for every row, the 16-byte blocks that cover its clamp-free source span,
// fetched with asynchronous 16-byte copies (no registers held while in flight; two buffers,
// so one batch's copies fly while the previous batch is written).  Then the CTA writes the
// batch's destination bytes, which are contiguous in the brick: as 16-byte blocks when
// rows and spans are 16-byte aligned and unclamped; as words on fixed (row, word) lane
// slots when rows are whole words and the slots keep most lanes busy; else as one run of
// words over the batch.  A word inside a row's span is one funnel shift of two staged
// words; words that touch the clamped columns or straddle two rows are assembled byte by
// byte.  Every brick byte maps to a staged byte: the clamped columns repeat the span's
// first or last voxel.
constexpr int ST_BUDGET = 24 * 1024;   // staged bytes per CTA (both buffers)
constexpr int ST_MAXROWS = 256;        // rows per batch (a multiple of 4)

__device__ __forceinline__ void cp_async16(uint32_t smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_group1()
{
    asm volatile("cp.async.wait_group 1;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// ES: bytes per voxel.  rows_per_cta and rb (rows per staged batch) are multiples of 4, so a
// batch's first destination byte is 4-byte aligned; pitch: staged bytes per row (a multiple
// of 16, at least 16 more than the widest span's covering blocks need).  Shared memory: two
// buffers of rb x pitch bytes.
// Off: the type of source byte offsets (uint32_t for volumes below 2^31 bytes).  BLK: every
// brick of the launch is written by 16-byte blocks (only that path is compiled in, which
// keeps registers and so occupancy for it).
template <int ES, typename Off, bool BLK>
__global__ void __launch_bounds__(NT, BLK ? 6 : 5)
    k_bricks_staged(const unsigned char* __restrict__ src, uint64_t vol_bytes, const BrickPtrs P,
                    const BrickGrid G, int rows_per_cta, int rb, int pitch)
{
    extern __shared__ __align__(16) unsigned char st[];
    __shared__ int s_shift[2][ST_MAXROWS];
    const int nx = G.nx, ny = G.ny, nz = G.nz, ghost = G.ghost;
    const BrickDesc b = brick_at(P, G);
    const int rows = b.dy * b.dz;
    const int r0 = blockIdx.x * rows_per_cta;
    if (r0 >= rows) return;
    const int r1 = min(rows, r0 + rows_per_cta);
    const int tid = threadIdx.x;
    const int sx0 = b.ox - ghost;
    const int left = clampd(-sx0, 0, b.dx);
    const int right = clampd(nx - sx0, left, b.dx);
    const int nb = (right - left) * ES;                 // span bytes (at least one voxel)
    const int lb = left * ES, rbyte = right * ES;       // span within the brick row, bytes
    const int L = b.dx * ES;                            // brick row bytes
    const int nv = (nb + 30) / 16;                      // covering blocks, any alignment
    const Off sb = static_cast<Off>(sx0 + left) * ES;
    unsigned char* dst = static_cast<unsigned char*>(b.dst);
    // the thread's words advance by 4 NT bytes: DR rows and DC bytes
    const int DR = (4 * NT) / L, DC = (4 * NT) - DR * L;

    // stage the spans of rows q0 .. q0 + nr - 1 into buffer buf (one async-copy group)
    // lanes of a warp take (row, block) slots: rpw rows of nv blocks per warp pass when the
    // blocks fit in a warp, else one row with the lanes striding over its blocks
    const int warp = tid >> 5, lane = tid & 31;
    const int rpw = nv <= 32 ? 32 / nv : 1;
    const int lrow = nv <= 32 ? lane / nv : 0;
    const int lv0 = nv <= 32 ? lane - lrow * nv : lane;
    const int rstep = NWARP * rpw;
    // the same slots for writing: 16-byte blocks (v16) or words of a row
    const bool v16 = lb == 0 && rbyte == L && (L & 15) == 0 && ((nx * ES) & 15) == 0 && (sb & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
    const int vpr16 = L >> 4, wpr4 = L >> 2;
    const int rpw16 = vpr16 >= 1 && vpr16 <= 32 ? 32 / vpr16 : 1;
    const int lrow16 = vpr16 >= 1 && vpr16 <= 32 ? lane / vpr16 : 0;
    const int lv16 = vpr16 >= 1 && vpr16 <= 32 ? lane - lrow16 * vpr16 : lane;
    const int rpw4 = wpr4 >= 1 && wpr4 <= 32 ? 32 / wpr4 : 1;
    const int lrow4 = wpr4 >= 1 && wpr4 <= 32 ? lane / wpr4 : 0;
    const int lw4 = wpr4 >= 1 && wpr4 <= 32 ? lane - lrow4 * wpr4 : lane;
    const bool words = (L & 3) == 0 && (wpr4 <= 32 ? 4 * rpw4 * wpr4 >= 3 * 32
                                                   : 4 * wpr4 >= 3 * 32 * ((wpr4 + 31) / 32));
    // 16-byte groups: rows of whole words and a 16-byte aligned brick (batches start at row
    // multiples of 4, so at multiples of 16 bytes); a thread's groups advance by 16 NT bytes
    const bool g16 = (L & 3) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
    const int DR16 = (16 * NT) / L, DC16 = (16 * NT) - DR16 * L;
    auto stage = [&](int q0, int nr, int buf) {
        const int boff = buf * rb * pitch;
        const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(st)) + boff;
        int* sh = s_shift[buf];
        int rr = warp * rpw + lrow;
        if (lrow >= rpw || rr >= nr) {
            cp_async_commit();
            return;
        }
        int k = (q0 + rr) / b.dy, j = q0 + rr - k * b.dy;
        for (; rr < nr; rr += rstep) {
            const int sz = clampd(b.oz - ghost + k, 0, nz - 1);
            const int sy = clampd(b.oy - ghost + j, 0, ny - 1);
            const Off a = (static_cast<Off>(sz) * ny + sy) * nx * ES + sb;
            const Off a16 = a & ~Off(15);
            if (lv0 == 0) sh[rr] = static_cast<int>(a - a16);
            for (int v = lv0; v < nv; v += 32) {
                const Off g = a16 + 16u * v;
                if (g >= a + nb) break;                 // past the span (smaller shift)
                const int so = rr * pitch + 16 * v;
                if (static_cast<uint64_t>(g) + 16 <= vol_bytes) {
                    cp_async16(sbase + so, src + g);
                } else {
                    for (int e = 0; e < 16; ++e)
                        if (static_cast<uint64_t>(g) + e < vol_bytes) st[boff + so + e] = src[g + e];
                }
            }
            j += rstep;
            while (j >= b.dy) {
                j -= b.dy;
                ++k;
            }
        }
        cp_async_commit();
    };

    // two buffers: the next batch's copies are in flight while this batch is written
    stage(r0, min(rb, r1 - r0), 0);
    for (int q0 = r0, buf = 0; q0 < r1; q0 += rb, buf ^= 1) {
        const int nr = min(rb, r1 - q0);
        if (q0 + rb < r1) {
            stage(q0 + rb, min(rb, r1 - q0 - rb), buf ^ 1);
            cp_async_wait_group1();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        const int boff = buf * rb * pitch;                 // buffer start in st (16-aligned)
        const uint32_t* sw = reinterpret_cast<const uint32_t*>(st + boff);
        const int* s_sh = s_shift[buf];
        // brick bytes [q0 L, (q0 + nr) L); byte c of batch row rr comes from staged byte
        // pos(c) of that row
        unsigned char* d0 = dst + static_cast<int64_t>(q0) * L;
        if (BLK || v16) {
            // whole rows, every span 16-byte aligned: 16-byte copies, lanes on (row, block)
            // slots as in the staging
            const uint4* s4 = reinterpret_cast<const uint4*>(st + boff);
            uint4* d4 = reinterpret_cast<uint4*>(d0);
            const int vpr = L >> 4;
            for (int r = warp * rpw16 + lrow16; lrow16 < rpw16 && r < nr; r += NWARP * rpw16)
                for (int v = lv16; v < vpr; v += 32) d4[r * vpr + v] = s4[(r * pitch >> 4) + v];
        } else if constexpr (BLK) {
            // not reached: BLK launches hold only block-copyable bricks
        } else if (words) {
            // rows of whole words, slots keeping at least 3/4 of the lanes busy: lanes on
            // (row, word) slots
            const int wpr = L >> 2;
            uint32_t* dw = reinterpret_cast<uint32_t*>(d0);
            for (int r = warp * rpw4 + lrow4; lrow4 < rpw4 && r < nr; r += NWARP * rpw4) {
                const int sh = s_sh[r];
                for (int w = lw4; w < wpr; w += 32) {
                    const int col = 4 * w;
                    uint32_t v;
                    if (col >= lb && col + 4 <= rbyte) {
                        const int bo = r * pitch + sh + (col - lb);
                        v = __funnelshift_r(sw[bo >> 2], sw[(bo >> 2) + 1], 8u * static_cast<uint32_t>(bo & 3));
                    } else {
                        v = 0;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int c = col + e;
                            const int pos = c < lb ? c % ES : (c >= rbyte ? nb - ES + (c - rbyte) % ES : c - lb);
                            v |= uint32_t(st[boff + r * pitch + sh + pos]) << (8 * e);
                        }
                    }
                    __stwb(dw + r * wpr + w, v);
                }
            }
        } else if (g16) {
            // rows of whole words, 16-byte aligned batches: the batch's bytes as one run of
            // 16-byte groups of four words (a group may span rows, a word may not)
            const int nbytes = nr * L;
            uint4* d4 = reinterpret_cast<uint4*>(d0);
            int rr = (16 * tid) / L, col = 16 * tid - rr * L;
            for (int g = tid; 16 * g < nbytes; g += NT) {
                uint32_t v[4];
                int r = rr, c = col;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (c >= L) {
                        c -= L;
                        ++r;
                    }
                    v[e] = 0;
                    if (16 * g + 4 * e < nbytes) {
                        const int sh = s_sh[r];
                        if (c >= lb && c + 4 <= rbyte) {
                            const int bo = r * pitch + sh + (c - lb);
                            v[e] = __funnelshift_r(sw[bo >> 2], sw[(bo >> 2) + 1],
                                                   8u * static_cast<uint32_t>(bo & 3));
                        } else {
#pragma unroll
                            for (int b2 = 0; b2 < 4; ++b2) {
                                const int cb = c + b2;
                                const int pos = cb < lb ? cb % ES
                                                        : (cb >= rbyte ? nb - ES + (cb - rbyte) % ES : cb - lb);
                                v[e] |= uint32_t(st[boff + r * pitch + sh + pos]) << (8 * b2);
                            }
                        }
                    }
                    c += 4;
                }
                if (16 * g + 16 <= nbytes) {
                    d4[g] = make_uint4(v[0], v[1], v[2], v[3]);
                } else {
                    uint32_t* dw = reinterpret_cast<uint32_t*>(d4 + g);
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (16 * g + 4 * e < nbytes) __stwb(dw + e, v[e]);
                }
                col += DC16;
                rr += DR16;
                while (col >= L) {
                    col -= L;
                    ++rr;
                }
            }
        } else {
        // rows of any length: the batch's bytes as one run of words (a word may straddle
        // two rows)
        const int nbytes = nr * L;
        uint32_t* dw = reinterpret_cast<uint32_t*>(d0);
        int rr = (4 * tid) / L, col = 4 * tid - rr * L;
        for (int w = tid; 4 * w < nbytes; w += NT) {
            uint32_t v;
            if (col >= lb && col + 4 <= rbyte) {
                const int bo = rr * pitch + s_sh[rr] + (col - lb);
                v = __funnelshift_r(sw[bo >> 2], sw[(bo >> 2) + 1], 8u * static_cast<uint32_t>(bo & 3));
            } else {
                int r = rr, c = col;
                v = 0;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (c >= L) {
                        c -= L;
                        ++r;
                    }
                    if (4 * w + e < nbytes) {
                        const int pos = c < lb ? c % ES : (c >= rbyte ? nb - ES + (c - rbyte) % ES : c - lb);
                        v |= uint32_t(st[boff + r * pitch + s_sh[r] + pos]) << (8 * e);
                    }
                    ++c;
                }
            }
            if (4 * w + 4 <= nbytes) {
                __stwb(dw + w, v);
            } else {
                unsigned char* d8 = reinterpret_cast<unsigned char*>(dw + w);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (4 * w + e < nbytes) d8[e] = static_cast<unsigned char>(v >> (8 * e));
            }
            col += DC;
            rr += DR;
            if (col >= L) {
                col -= L;
                ++rr;
            }
        }
        }
        __syncthreads();   // buffer buf is refilled by the batch after next
    }
}

// Plane-image variant, for ghost cells on a source a tensor map describes.  Brick plane k
// (source plane clamp(oz - ghost + k)) is one contiguous run of dx * dy voxels in the brick,
// and the source voxels it needs lie in one box: columns [ox - XA, ox + bx + XA) (XA = 16
// bytes of voxels, so the box starts on a 16-byte boundary and holds ghost <= XA columns on
// either side), rows [oy - ghost, oy + by + ghost).  A CTA takes a run of one brick's planes:
// TMA brings each plane's box into a ring of stages (rows and columns outside the volume
// arrive zero-filled, the z coordinate is clamped), and the threads write the brick plane as
// words, lanes on consecutive words (one 128-byte store per warp): word c of brick row j is
// staged row clamp(oy - ghost + j) - (oy - ghost), bytes (XA - ghost) * ES + 4c onward, one
// funnel shift of two staged words (the shift is the same for every word of the launch).
// Bricks whose ghost columns reach past an x face of the volume assemble each word voxel by
// voxel from clamped columns instead.  Needs brick rows of whole words (dx * ES a multiple
// of 4), 4-byte aligned bricks, and bx * ES a multiple of 16 (box starts on 16-byte
// boundaries).  Every wait is bounded; on a timeout the CTA records it and drains its loads.
constexpr int PL_STAGES = 4;

struct PlaneArgs {
    int ppc;             // brick planes per CTA
    int boxw, boxh;      // box extent (voxels, rows)
    int stage;           // bytes per stage (box bytes rounded up, with 16 bytes of slack)
    uint32_t txb;        // bytes one box delivers
    unsigned* status;
};

template <int ES>
__global__ void __launch_bounds__(NT)
    k_bricks_planes(const __grid_constant__ CUtensorMap tmap, const BrickPtrs P, const BrickGrid G,
                    const PlaneArgs A)
{
    constexpr int XA = 16 / ES;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    unsigned char* ring = smem + 128;
    const BrickDesc b = brick_at(P, G);
    const int g = G.ghost;
    const int k0 = blockIdx.x * A.ppc;
    if (k0 >= b.dz) return;
    const int np = min(b.dz, k0 + A.ppc) - k0;
    const int tid = threadIdx.x;
    const int rb = A.boxw * ES;                  // staged row bytes
    const int wpr = (b.dx * ES) >> 2;            // words per brick row
    const int nwords = wpr * b.dy;               // words per brick plane
    const int bx0 = b.ox - XA, by0 = b.oy - g;   // box origin
    const bool xin = b.ox - g >= 0 && b.ox + b.dx - g <= G.nx;
    const bool yin = by0 >= 0 && by0 + b.dy <= G.ny;
    if (tid == 0) {
        for (int q = 0; q < PL_STAGES; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
        prefetch_tensor_map(&tmap);
    }
    __syncthreads();
    int issued = 0;   // planes handed to the TMA unit (thread 0 only)
    auto issue = [&](int q) {
        const int s = q % PL_STAGES;
        mbar_arrive_expect_tx(&bars[s], A.txb);
        tma_load_3d(ring + s * A.stage, &tmap, &bars[s], bx0, by0,
                    clampi(b.oz - g + k0 + q, 0, G.nz - 1));
        ++issued;
    };
    if (tid == 0)
        for (int q = 0; q < PL_STAGES && q < np; ++q) issue(q);
    // the thread's words advance by NT words: DR rows and DC words
    const int DR = NT / wpr, DC = NT - DR * wpr;
    const int r0 = tid / wpr, c0 = tid - r0 * wpr;
    const int off0 = (XA - g) * ES;               // staged byte of brick column 0
    const uint32_t sh = 8u * static_cast<uint32_t>(off0 & 3);
    uint32_t* dst = static_cast<uint32_t*>(b.dst);
    bool failed = false;
    for (int q = 0; q < np; ++q) {
        const int s = q % PL_STAGES;
        const bool ok = mbar_wait(&bars[s], (q / PL_STAGES) & 1);
        if (ok) {
            const unsigned char* st = ring + s * A.stage;
            const uint32_t* sw = reinterpret_cast<const uint32_t*>(st);
            uint32_t* dp = dst + static_cast<int64_t>(k0 + q) * nwords;
            int r = r0, c = c0;
            for (int w = tid; w < nwords; w += NT) {
                const int sr = yin ? r : clampi(by0 + r, 0, G.ny - 1) - by0;
                uint32_t v;
                if (xin) {
                    const int bo = sr * rb + off0 + 4 * c;
                    v = __funnelshift_r(sw[bo >> 2], sw[(bo >> 2) + 1], sh);
                } else {
                    v = 0;
#pragma unroll
                    for (int e = 0; e < 4 / ES; ++e) {
                        const int x = clampi(b.ox - g + (4 / ES) * c + e, 0, G.nx - 1);
                        const unsigned char* sp = st + sr * rb + (x - bx0) * ES;
                        const uint32_t t = ES == 1 ? *sp
                                         : ES == 2 ? *reinterpret_cast<const uint16_t*>(sp)
                                                   : *reinterpret_cast<const uint32_t*>(sp);
                        v |= t << (8 * ES * e);
                    }
                }
                __stcs(dp + w, v);
                c += DC;
                r += DR;
                if (c >= wpr) {
                    c -= wpr;
                    ++r;
                }
            }
        }
        // every thread is done with stage s: it takes plane q + PL_STAGES
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (tid == 0 && q + PL_STAGES < np) issue(q + PL_STAGES);
    }
    if (failed && tid == 0) {
        atomicOr(A.status, STATUS_TIMEOUT);
        for (int q = issued - 1; q >= 0 && q >= issued - PL_STAGES; --q)
            mbar_wait(&bars[q % PL_STAGES], (q / PL_STAGES) & 1);
    }
}

int bricks_along(int n, int b) { return (n + b - 1) / b; }

// The plane-image kernel over every brick of a call (the caller checked its conditions and
// encoded the tensor map with a box of (bx + 2 XA) x (by + 2 ghost) x 1 voxels).
vktError launch_planes(const vktStructuredVolume* bricks, int numBricks, const BrickGrid& G0,
                       int es, const CUtensorMap& map, int max_dz, const Ctx& ctx, int sms,
                       int* launches)
{
    const int xa = 16 / es;
    PlaneArgs A;
    A.boxw = G0.bx + 2 * xa;
    A.boxh = G0.by + 2 * G0.ghost;
    A.txb = static_cast<uint32_t>(A.boxw) * es * A.boxh;
    A.stage = static_cast<int>((A.txb + 16 + 127) & ~127u);
    A.status = ctx.status;
    const size_t smem = 128 + static_cast<size_t>(PL_STAGES) * A.stage;
    const void* kern = es == 1 ? reinterpret_cast<const void*>(k_bricks_planes<1>)
                     : es == 2 ? reinterpret_cast<const void*>(k_bricks_planes<2>)
                               : reinterpret_cast<const void*>(k_bricks_planes<4>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return from_cuda(e);
    // planes per CTA for whole waves of the resident CTAs: the least waves x (planes per CTA
    // + 2, a CTA's set-up counted as planes)
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess)
        per_sm = 1;
    const int64_t slots = static_cast<int64_t>(sms) * std::max(per_sm, 1);
    int64_t best = -1;
    A.ppc = max_dz;
    for (int c = 1; c <= max_dz; ++c) {
        const int ppc = (max_dz + c - 1) / c;
        const int64_t ctas = static_cast<int64_t>((max_dz + ppc - 1) / ppc) * numBricks;
        const int64_t cost = ((ctas + slots - 1) / slots) * (ppc + 2);
        if (best < 0 || cost < best) {
            best = cost;
            A.ppc = ppc;
        }
    }
    const int gx = (max_dz + A.ppc - 1) / A.ppc;
    BrickGrid G = G0;
    std::unique_ptr<BrickPtrs> P(new BrickPtrs);
    for (int first = 0; e == cudaSuccess && first < numBricks; first += MAXB) {
        const int nb = std::min(MAXB, numBricks - first);
        for (int i = 0; i < nb; ++i) P->p[i] = bricks[first + i]->data;
        G.first = first;
        const dim3 grid(gx, nb);
        if (es == 1)
            k_bricks_planes<1><<<grid, NT, smem, ctx.stream>>>(map, *P, G, A);
        else if (es == 2)
            k_bricks_planes<2><<<grid, NT, smem, ctx.stream>>>(map, *P, G, A);
        else
            k_bricks_planes<4><<<grid, NT, smem, ctx.stream>>>(map, *P, G, A);
        e = cudaGetLastError();
        ++*launches;
    }
    if (ctx.debug & VKT_DEBUG_LOG)
        fprintf(stderr, "[vkt] brick-decompose %d bricks (%dx%dx%d, ghost %d) grid=(%d,%d) planes=%d planes launches=%d\n",
                numBricks, G0.bx, G0.by, G0.bz, G0.ghost, gx, std::min(numBricks, MAXB), A.ppc, *launches);
    return from_cuda(e);
}

}  // namespace
}  // namespace vkt

using namespace vkt;

extern "C" {

vktError vktBrickDecomposeCountSV(int32_t* countX, int32_t* countY, int32_t* countZ,
                                  vktStructuredVolume volume, int32_t brickX, int32_t brickY,
                                  int32_t brickZ)
{
    if (!valid_volume(volume)) return VKT_ERROR_INVALID_HANDLE;
    if (!countX || !countY || !countZ || brickX < 1 || brickY < 1 || brickZ < 1)
        return VKT_ERROR_INVALID_VALUE;
    *countX = bricks_along(volume->dims[0], brickX);
    *countY = bricks_along(volume->dims[1], brickY);
    *countZ = bricks_along(volume->dims[2], brickZ);
    return VKT_NO_ERROR;
}

vktError vktBrickDecomposeSV(vktStructuredVolume* bricks, int32_t numBricks,
                             vktStructuredVolume volume, int32_t brickX, int32_t brickY,
                             int32_t brickZ, int32_t ghost)
{
    vkt::CallRange nvtx_range("vktBrickDecomposeSV");
    if (!valid_volume(volume)) return VKT_ERROR_INVALID_HANDLE;
    if (!bricks || brickX < 1 || brickY < 1 || brickZ < 1 || ghost < 0)
        return VKT_ERROR_INVALID_VALUE;
    const int nx = volume->dims[0], ny = volume->dims[1], nz = volume->dims[2];
    const int b[3] = {brickX, brickY, brickZ};
    const int cx = bricks_along(nx, brickX), cy = bricks_along(ny, brickY), cz = bricks_along(nz, brickZ);
    if (static_cast<int64_t>(cx) * cy * cz != numBricks) return VKT_ERROR_INVALID_VALUE;
    const int es = elem_bytes(volume->format);
    const char* s0 = static_cast<const char*>(volume->data);
    const uint64_t sbytes = static_cast<uint64_t>(nx) * ny * nz * es;
    int max_rows = 0, pitch = 0;
    bool staged = (reinterpret_cast<uintptr_t>(volume->data) & 15) == 0;
    for (int kz = 0; kz < cz; ++kz)
        for (int ky = 0; ky < cy; ++ky)
            for (int kx = 0; kx < cx; ++kx) {
                const size_t i = (static_cast<size_t>(kz) * cy + ky) * cx + kx;
                const vktStructuredVolume_impl* v = bricks[i];
                if (!valid_volume(v)) return VKT_ERROR_INVALID_HANDLE;
                if (v->format != volume->format) return VKT_ERROR_INVALID_VALUE;
                const int o[3] = {kx * b[0], ky * b[1], kz * b[2]};
                const int n[3] = {nx, ny, nz};
                int dd[3];
                for (int a = 0; a < 3; ++a) dd[a] = std::min(b[a], n[a] - o[a]) + 2 * ghost;
                if (v->dims[0] != dd[0] || v->dims[1] != dd[1] || v->dims[2] != dd[2])
                    return VKT_ERROR_DIMS_MISMATCH;
                const char* p = static_cast<const char*>(v->data);
                const uint64_t bytes = static_cast<uint64_t>(dd[0]) * dd[1] * dd[2] * es;
                if (p < s0 + sbytes && s0 < p + bytes) return VKT_ERROR_INVALID_VALUE;
                max_rows = std::max(max_rows, dd[1] * dd[2]);
                // staged kernel: 4-byte aligned bricks; staged bytes per row for the span
                staged = staged && (reinterpret_cast<uintptr_t>(v->data) & 3) == 0;
                const int sx0 = o[0] - ghost;
                const int left = std::min(std::max(-sx0, 0), dd[0]);
                const int right = std::min(std::max(nx - sx0, left), dd[0]);
                pitch = std::max(pitch, ((right - left) * es + 30) / 16 * 16 + 16);
            }
    Ctx ctx;
    vktError err = get_context(&ctx);
    if (err != VKT_NO_ERROR) return err;
    // rows per CTA: enough that the grid is a few waves (short brick rows make small CTAs
    // latency-bound), at least MIN_ROWS_PER_CTA
    int sms = 152;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int64_t total_rows = static_cast<int64_t>(max_rows) * numBricks;
    const int64_t want = std::max<int64_t>(MIN_ROWS_PER_CTA, total_rows / (static_cast<int64_t>(sms) * 32));
    int rows_per_cta = static_cast<int>(std::min<int64_t>(want, max_rows));
    // staged batches must hold at least 4 rows
    int rb = std::min(ST_MAXROWS, (ST_BUDGET / (2 * std::max(pitch, 1))) & ~3);
    staged = staged && rb >= 4;
    // every brick block-copyable: no ghost cells, rows and brick widths (the last one along x
    // included) multiples of 16 bytes, bricks 16-byte aligned
    bool blk = staged && ghost == 0 && (static_cast<int64_t>(nx) * es) % 16 == 0 &&
               (static_cast<int64_t>(brickX) * es) % 16 == 0 &&
               (static_cast<int64_t>(nx - (cx - 1) * brickX) * es) % 16 == 0;
    for (int i = 0; blk && i < numBricks; ++i) blk = (reinterpret_cast<uintptr_t>(bricks[i]->data) & 15) == 0;
    const bool small = sbytes < (uint64_t(1) << 31);
    const void* skern = nullptr;
    if (staged) {
#define VKT_PICK(E)                                                                             \
    skern = small ? (blk ? reinterpret_cast<const void*>(k_bricks_staged<E, uint32_t, true>)    \
                         : reinterpret_cast<const void*>(k_bricks_staged<E, uint32_t, false>)) \
                  : (blk ? reinterpret_cast<const void*>(k_bricks_staged<E, uint64_t, true>)    \
                         : reinterpret_cast<const void*>(k_bricks_staged<E, uint64_t, false>))
        if (es == 1) VKT_PICK(1); else if (es == 2) VKT_PICK(2); else VKT_PICK(4);
#undef VKT_PICK
        // rows per CTA for whole waves of the resident CTAs: the least waves x (rows per CTA
        // + 32, a CTA's fixed setup counted as rows) over 1 to 64 runs per brick (multiples
        // of 4 rows, at least MIN_ROWS_PER_CTA)
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, skern, NT,
                                                          2 * static_cast<size_t>(rb) * pitch) != cudaSuccess)
            per_sm = 1;
        const int64_t slots = static_cast<int64_t>(sms) * std::max(per_sm, 1);
        int64_t best = -1;
        for (int c = 1; c <= 64; ++c) {
            const int rpc = std::max(std::min(MIN_ROWS_PER_CTA, (max_rows + 3) & ~3),
                                     (((max_rows + c - 1) / c) + 3) & ~3);
            const int64_t ctas = static_cast<int64_t>((max_rows + rpc - 1) / rpc) * numBricks;
            const int64_t cost = ((ctas + slots - 1) / slots) * (rpc + 32);
            if (best < 0 || cost < best) {
                best = cost;
                rows_per_cta = rpc;
            }
        }
        rb = std::min(rb, rows_per_cta);
    }
    BrickGrid G;
    G.nx = nx;
    G.ny = ny;
    G.nz = nz;
    G.bx = brickX;
    G.by = brickY;
    G.bz = brickZ;
    G.cx = cx;
    G.cy = cy;
    G.ghost = ghost;
    // ghost cells on a source a tensor map describes: the plane-image kernel, when the brick
    // width starts every box on a 16-byte boundary, the ghosts fit the box's 16-byte x halo,
    // the bricks are 4-byte aligned with rows of whole words, and the ring fits shared memory
    {
        const int pxa = 16 / es;
        bool planes = ghost >= 1 && ghost <= pxa && (static_cast<int64_t>(brickX) * es) % 16 == 0 &&
                      brickX + 2 * pxa <= 256 && brickY + 2 * ghost <= 256 &&
                      static_cast<int64_t>(brickX + 2 * pxa) * es * (brickY + 2 * ghost) <= 40 * 1024;
        int max_dz = 0;
        for (int i = 0; planes && i < numBricks; ++i) {
            planes = (reinterpret_cast<uintptr_t>(bricks[i]->data) & 3) == 0 &&
                     (static_cast<int64_t>(bricks[i]->dims[0]) * es) % 4 == 0;
            max_dz = std::max(max_dz, bricks[i]->dims[2]);
        }
        alignas(64) CUtensorMap pmap;
        if (planes)
            planes = encode_tensor_map_3d(&pmap, volume->format, volume->data, nx, ny, nz,
                                          brickX + 2 * pxa, brickY + 2 * ghost, 1);
        if (planes) {
            int launches = 0;
            const vktError pe = launch_planes(bricks, numBricks, G, es, pmap, max_dz, ctx, sms, &launches);
            count_launches(launches);
            return pe;
        }
    }
    const int gx = (max_rows + rows_per_cta - 1) / rows_per_cta;
    std::unique_ptr<BrickPtrs> P(new BrickPtrs);
    cudaError_t e = cudaSuccess;
    int launches = 0;
    for (int first = 0; e == cudaSuccess && first < numBricks; first += MAXB) {
        const int nb = std::min(MAXB, numBricks - first);
        for (int i = 0; i < nb; ++i) P->p[i] = bricks[first + i]->data;
        G.first = first;
        const dim3 grid(gx, nb);
        const unsigned char* s8 = static_cast<const unsigned char*>(volume->data);
        if (staged) {
            const size_t sm = 2 * static_cast<size_t>(rb) * pitch;
#define VKT_BRICKS_STAGED(E, O)                                                                      \
    (blk ? k_bricks_staged<E, O, true> : k_bricks_staged<E, O, false>)<<<grid, NT, sm, ctx.stream>>>( \
        s8, sbytes, *P, G, rows_per_cta, rb, pitch)
            if (es == 1) {
                if (small) VKT_BRICKS_STAGED(1, uint32_t); else VKT_BRICKS_STAGED(1, uint64_t);
            } else if (es == 2) {
                if (small) VKT_BRICKS_STAGED(2, uint32_t); else VKT_BRICKS_STAGED(2, uint64_t);
            } else {
                if (small) VKT_BRICKS_STAGED(4, uint32_t); else VKT_BRICKS_STAGED(4, uint64_t);
            }
#undef VKT_BRICKS_STAGED
        } else if (es == 1) {
            k_bricks<uint8_t><<<grid, NT, 0, ctx.stream>>>(static_cast<const uint8_t*>(volume->data), *P, G,
                                                           rows_per_cta);
        } else if (es == 2) {
            k_bricks<uint16_t><<<grid, NT, 0, ctx.stream>>>(static_cast<const uint16_t*>(volume->data), *P, G,
                                                            rows_per_cta);
        } else {
            k_bricks<uint32_t><<<grid, NT, 0, ctx.stream>>>(static_cast<const uint32_t*>(volume->data), *P, G,
                                                            rows_per_cta);
        }
        e = cudaGetLastError();
        ++launches;
    }
    count_launches(launches);
    if (ctx.debug & VKT_DEBUG_LOG)
        fprintf(stderr, "[vkt] brick-decompose %d bricks (%dx%dx%d, ghost %d) grid=(%d,%d) %s launches=%d\n",
                numBricks, brickX, brickY, brickZ, ghost, gx, std::min(numBricks, MAXB),
                staged ? (blk ? "staged blocks" : "staged") : "plain", launches);
    return from_cuda(e);
}

}  // extern "C"
