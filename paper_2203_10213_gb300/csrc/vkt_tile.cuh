// vkt_tile.cuh -- device helpers shared by the filter kernels: mbarrier and TMA wrappers
// (inline PTX, sm_103a), bounded waits, brick geometry, the raw-tile to float-tile
// conversion with clamp-to-edge, and the output epilogue.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace vkt {

enum : int { FMT_U8 = 0, FMT_U16 = 1, FMT_F32 = 2 };

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;   // 2 s for any single device wait

__host__ __device__ constexpr int fmt_bytes(int f) { return f == FMT_U8 ? 1 : (f == FMT_U16 ? 2 : 4); }
// TMA needs the innermost start coordinate on a 16-byte boundary: x halo per side
__host__ __device__ constexpr int fmt_xalign(int f) { return 16 / fmt_bytes(f); }

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// bytes of dynamic shared memory this CTA was launched with
__device__ __forceinline__ uint32_t dynamic_smem_bytes()
{
    uint32_t v;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}

// Programmatic dependent launch.  A kernel launched with programmatic stream serialization
// (launch_pdl) may begin while the kernel before it on the stream is still running: it sets
// up its shared memory and barriers, then waits in grid_dependency_wait() until that kernel
// has completed and its writes are visible, before its first global-memory access.
// launch_dependents() lets the next such kernel begin its own set-up once every CTA of this
// grid is running.
__device__ __forceinline__ void grid_dependency_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// orders this thread's generic-proxy writes to shared memory before later async-proxy
// (TMA) writes to the same bytes
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait that lets the thread be suspended (up to the hint, in ns) until the phase
// completes, instead of returning at once; waiting warps then leave their issue slots to
// the others on the sub-partition
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

// Waits for the phase of `parity` to complete; false after WAIT_LIMIT_NS.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait_sleep(bar, parity)) {
        if (global_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
    return true;
}

// 3-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// 4-D tiled TMA load (x, y, z, volume of a batch) of one box into shared memory.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z, int v)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(v), "r"(smem_u32(bar))
        : "memory");
}

// 1-D bulk copy global -> shared (both addresses 16-byte aligned, bytes a multiple of 16)
// completing `bytes` transactions on the mbarrier
__device__ __forceinline__ void bulk_load_1d(void* dst, const void* src, uint32_t bytes,
                                             uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes),
        "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tensor_map(const CUtensorMap* map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// Geometry of one brick plane: TX x TY outputs, radius R, float tile of (TY+2R) rows
// starting at (x0-R, y0-R), pitch a multiple of 4 floats.  The raw tile (what TMA
// writes) starts at (x0 - XA, y0 - R), with XA = 16 bytes / voxel size >= R.
template <int K, int TX, int TY>
struct Brick {
    static constexpr int R = (K - 1) / 2;
    static constexpr int FW = TX + 2 * R;
    static constexpr int FP = (FW + 3) & ~3;
    static constexpr int FH = TY + 2 * R;
    static constexpr int FGROUPS = FP / 4;          // float4 groups per row
    static_assert(R <= 4, "x halo of a float32 raw tile is 4 voxels");
    __host__ __device__ static constexpr int raw_w(int fmt) { return TX + 2 * fmt_xalign(fmt); }
    // bytes one TMA box delivers
    __host__ __device__ static constexpr int raw_tx(int fmt) { return raw_w(fmt) * FH * fmt_bytes(fmt); }
    // row pitch (bytes) of a stage filled by row copies: a raw row plus up to 15 bytes of
    // 16-byte misalignment in front of it
    __host__ __device__ static constexpr int row_pitch(int fmt) { return raw_w(fmt) * fmt_bytes(fmt) + 16; }
    // the (128-byte padded) size of one raw stage filled by a TMA box or plain loads, and of
    // one filled by row copies
    __host__ __device__ static constexpr int raw_bytes(int fmt) { return (raw_tx(fmt) + 127) & ~127; }
    __host__ __device__ static constexpr int rows_bytes(int fmt) { return (FH * row_pitch(fmt) + 127) & ~127; }
    __host__ __device__ static constexpr int stage_bytes(int fmt, bool rows)
    {
        return rows ? rows_bytes(fmt) : raw_bytes(fmt);
    }
};

// Row-copy loading, for volumes whose rows are not a multiple of 16 bytes long (no tensor
// map can describe them).  Stage row r (r < FH, global row y0 - R + r inside the volume) is
// filled by one 1-D bulk copy of the 16-byte aligned span around raw columns
// [0, raw_w) = voxels [x0 - xa, x0 - xa + raw_w) of plane clamp(z); the raw column 0 of the
// row lands at the row's misalignment (row_shift_elems) in the stage row.  Rows outside the
// volume are not copied: the clamped conversion never reads them.  The copies are clipped
// to the volume's full 16-byte blocks, so no byte outside the volume is read; the few bytes
// of the last partial block a row needs are read with plain loads.
//
// Every thread of the CTA calls issue_rows; thread (lane l, warp w) takes row 8 l + w, so
// the rows spread over the warps.  Each copying thread first adds its bytes to the stage
// barrier's transaction count (expect_tx, no arrival), then starts its copy.  The caller
// makes the barrier's single arrival (rows_arrive) from one thread after a CTA barrier that
// follows every thread's issue_rows, so the phase cannot complete before all bytes are
// expected, and the plain-loaded bytes are visible to whoever waits on the phase.
__device__ __forceinline__ uint32_t row_shift_elems(uint32_t zterm, int gy, int nx, int x0, int xa,
                                                    int fmt)
{
    const uint32_t mask = static_cast<uint32_t>(16 / fmt_bytes(fmt)) - 1u;
    return (zterm + static_cast<uint32_t>(gy) * static_cast<uint32_t>(nx) +
            static_cast<uint32_t>(x0 - xa)) & mask;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

template <typename Geo, int NT>
__device__ __forceinline__ void issue_rows(unsigned char* stage, uint64_t* bar, const void* src,
                                           uint64_t vol_bytes, int fmt, int nx, int ny, int nz,
                                           int x0, int y0, int z, int tid)
{
    static_assert(NT % 32 == 0 && Geo::FH <= 32 * (NT / 32), "one row per thread at most");
    const int r = (tid & 31) * (NT / 32) + (tid >> 5);
    if (r >= Geo::FH) return;
    const int yy = y0 - Geo::R + r;
    if (yy < 0 || yy >= ny) return;
    const int es = fmt_bytes(fmt);
    const int xa = fmt_xalign(fmt);
    const int64_t need = static_cast<int64_t>(Geo::raw_w(fmt)) * es;
    const int64_t full = static_cast<int64_t>(vol_bytes & ~uint64_t(15));
    const int gz = clampi(z, 0, nz - 1);
    const unsigned char* base = static_cast<const unsigned char*>(src);
    const int64_t b0 = ((static_cast<int64_t>(gz) * ny + yy) * nx + (x0 - xa)) * es;
    const int64_t a0 = b0 - (b0 & 15);          // floor to 16 bytes (also for b0 < 0)
    const int64_t a1 = (b0 + need + 15) & ~int64_t(15);
    const int64_t lo = a0 > 0 ? a0 : 0;
    const int64_t hi = a1 < full ? a1 : full;
    unsigned char* row = stage + r * Geo::row_pitch(fmt);
    if (hi > lo) {
        mbar_expect_tx(bar, static_cast<uint32_t>(hi - lo));
        bulk_load_1d(row + (lo - a0), base + lo, static_cast<uint32_t>(hi - lo), bar);
    }
    // bytes past the last full block that this row needs
    const int64_t t1 = (b0 + need) < static_cast<int64_t>(vol_bytes) ? (b0 + need)
                                                                      : static_cast<int64_t>(vol_bytes);
    for (int64_t bb = (full > b0 ? full : b0); bb < t1; ++bb) row[bb - a0] = __ldg(base + bb);
}

// Fills the raw tile of plane z with plain loads (the path for volumes whose rows cannot
// be described by a tensor map).  Only the columns the conversion reads are written: raw
// columns [xa - R, xa + TX + R), i.e. voxels x0 - R .. x0 + TX + R - 1.  Each warp takes
// whole rows and its lanes consecutive columns, so the loads of a warp are coalesced and
// no index needs a division; a lane's loads of one row are issued together before their
// stores.  CLAMP: positions outside the volume receive the
// clamped neighbour (the conversion never reads them anyway); otherwise they receive zero,
// the zero extension the adjoint needs (and what a TMA load writes there).
template <typename Geo, int NT, bool CLAMP = true>
__device__ __forceinline__ void fill_raw_plain(unsigned char* raw, const void* src, int fmt,
                                               int nx, int ny, int nz, int x0, int y0, int z,
                                               int tid)
{
    constexpr int NW = NT / 32;
    constexpr int COLS = Geo::FW;
    const int xa = fmt_xalign(fmt);
    const int rw = Geo::raw_w(fmt);
    const int warp = tid >> 5, lane = tid & 31;
    const bool zin = z >= 0 && z < nz;
    const int64_t plane = static_cast<int64_t>(clampi(z, 0, nz - 1)) * nx * ny;
#pragma unroll 1
    for (int rr = 0; rr < (Geo::FH + NW - 1) / NW; ++rr) {
        const int row = warp + rr * NW;
        if (row >= Geo::FH) break;
        const int yy = y0 - Geo::R + row;
        const bool yin = zin && yy >= 0 && yy < ny;
        const int64_t rbase = plane + static_cast<int64_t>(clampi(yy, 0, ny - 1)) * nx;
        const int dbase = row * rw + xa - Geo::R;
        // a row's loads first (in flight together), then its shared-memory stores
        constexpr int NC = (COLS + 31) / 32;
        uint32_t v[NC];
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
            const int c = min(lane + cc * 32, COLS - 1);
            const int64_t gi = rbase + clampi(x0 - Geo::R + c, 0, nx - 1);
            if (fmt == FMT_F32)
                v[cc] = __float_as_uint(__ldg(reinterpret_cast<const float*>(src) + gi));
            else if (fmt == FMT_U16)
                v[cc] = __ldg(reinterpret_cast<const uint16_t*>(src) + gi);
            else
                v[cc] = __ldg(reinterpret_cast<const unsigned char*>(src) + gi);
        }
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
            const int c = lane + cc * 32;
            if (c >= COLS) break;
            const int xx = x0 - Geo::R + c;
            const uint32_t val = (CLAMP || (yin && xx >= 0 && xx < nx)) ? v[cc] : 0u;
            const int e = dbase + c;
            if (fmt == FMT_F32)
                reinterpret_cast<uint32_t*>(raw)[e] = val;
            else if (fmt == FMT_U16)
                reinterpret_cast<uint16_t*>(raw)[e] = static_cast<uint16_t>(val);
            else
                raw[e] = static_cast<unsigned char>(val);
        }
    }
}

// Per-thread precomputed raw-tile offsets of the float-tile groups this thread converts.
// Group gi covers float-tile row gi / FGROUPS, columns 4*(gi % FGROUPS) .. +3; each of
// its 4 elements reads the raw tile at the clamped voxel position.
template <typename Geo, int NT, bool CLAMP = true>
struct ConvPlan {
    static constexpr int NG = (Geo::FH * Geo::FGROUPS + NT - 1) / NT;
    int off[NG][4];

    // rows: the stage is filled by row copies (row pitch Geo::row_pitch), not by one TMA box
    __device__ __forceinline__ void init(int fmt, int nx, int ny, int x0, int y0, int tid,
                                         bool rows = false)
    {
        const int xa = fmt_xalign(fmt);
        const int rw = rows ? Geo::row_pitch(fmt) / fmt_bytes(fmt) : Geo::raw_w(fmt);
#pragma unroll
        for (int n = 0; n < NG; ++n) {
            const int gi = tid + n * NT;
            const int row = gi / Geo::FGROUPS;
            const int g = gi - row * Geo::FGROUPS;
            // CLAMP: the clamped voxel; otherwise the position itself (the raw tile holds
            // zeros outside the volume there)
            const int gy = CLAMP ? clampi(y0 - Geo::R + row, 0, ny - 1) : y0 - Geo::R + row;
            const int rrow = gy - (y0 - Geo::R);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                // padding columns past the halo repeat the last halo column
                const int j = min(4 * g + e, Geo::FW - 1);
                const int gx = CLAMP ? clampi(x0 - Geo::R + j, 0, nx - 1) : x0 - Geo::R + j;
                off[n][e] = rrow * rw + (gx - (x0 - xa));
            }
        }
    }

    // raw tile -> float tile (pitch FP), every element mapped to its clamped voxel
    __device__ __forceinline__ void convert(const unsigned char* raw, int fmt, float* F,
                                            int tid) const
    {
#pragma unroll
        for (int n = 0; n < NG; ++n) {
            const int gi = tid + n * NT;
            if (NG * NT > Geo::FH * Geo::FGROUPS && gi >= Geo::FH * Geo::FGROUPS) break;
            float4 v;
            if (fmt == FMT_F32) {
                const float* r = reinterpret_cast<const float*>(raw);
                v = make_float4(r[off[n][0]], r[off[n][1]], r[off[n][2]], r[off[n][3]]);
            } else if (fmt == FMT_U16) {
                const uint16_t* r = reinterpret_cast<const uint16_t*>(raw);
                v = make_float4(r[off[n][0]], r[off[n][1]], r[off[n][2]], r[off[n][3]]);
            } else {
                v = make_float4(raw[off[n][0]], raw[off[n][1]], raw[off[n][2]], raw[off[n][3]]);
            }
            reinterpret_cast<float4*>(F)[gi] = v;
        }
    }

    // the same for a stage filled by issue_rows (clamped conversion only): each row's
    // elements sit row_shift_elems() further in; zterm = clamp(z) * ny * nx (mod 2^32)
    __device__ __forceinline__ void convert_rows(const unsigned char* raw, int fmt, float* F,
                                                 int tid, int nx, int ny, int x0, int y0,
                                                 uint32_t zterm) const
    {
        static_assert(CLAMP, "row-copied stages hold only rows inside the volume");
        const int xa = fmt_xalign(fmt);
#pragma unroll
        for (int n = 0; n < NG; ++n) {
            const int gi = tid + n * NT;
            if (NG * NT > Geo::FH * Geo::FGROUPS && gi >= Geo::FH * Geo::FGROUPS) break;
            const int row = gi / Geo::FGROUPS;
            const int gy = clampi(y0 - Geo::R + row, 0, ny - 1);
            const int m = static_cast<int>(row_shift_elems(zterm, gy, nx, x0, xa, fmt));
            float4 v;
            if (fmt == FMT_F32) {
                const float* r = reinterpret_cast<const float*>(raw) + m;
                v = make_float4(r[off[n][0]], r[off[n][1]], r[off[n][2]], r[off[n][3]]);
            } else if (fmt == FMT_U16) {
                const uint16_t* r = reinterpret_cast<const uint16_t*>(raw) + m;
                v = make_float4(r[off[n][0]], r[off[n][1]], r[off[n][2]], r[off[n][3]]);
            } else {
                const unsigned char* r = raw + m;
                v = make_float4(r[off[n][0]], r[off[n][1]], r[off[n][2]], r[off[n][3]]);
            }
            reinterpret_cast<float4*>(F)[gi] = v;
        }
    }
};

// Loads N consecutive floats from shared memory aligned to VEC floats (VEC = 1, 2 or 4).
template <int N, int VEC>
__device__ __forceinline__ void load_row(const float* p, float (&v)[N])
{
    constexpr int N4 = (VEC == 4) ? (N / 4) * 4 : 0;
#pragma unroll
    for (int i = 0; i < N4; i += 4) {
        const float4 t = *reinterpret_cast<const float4*>(p + i);
        v[i] = t.x; v[i + 1] = t.y; v[i + 2] = t.z; v[i + 3] = t.w;
    }
    constexpr int N2 = (VEC >= 2) ? N4 + ((N - N4) / 2) * 2 : 0;
#pragma unroll
    for (int i = N4; i < N2; i += 2) {
        const float2 t = *reinterpret_cast<const float2*>(p + i);
        v[i] = t.x; v[i + 1] = t.y;
    }
#pragma unroll
    for (int i = N2; i < N; ++i) v[i] = p[i];
}

// Writes results first .. nvalid-1 of RX consecutive results of one row (from idx), mapped
// to the destination format.
template <int RX>
__device__ __forceinline__ void store_row(void* dst, int dfmt, int64_t idx, int nvalid,
                                          const float (&acc)[RX], float a0, float a1, float qmax,
                                          int first = 0)
{
    float v[RX];
#pragma unroll
    for (int x = 0; x < RX; ++x) v[x] = fmaf(a1, acc[x], a0);
    if (dfmt == FMT_F32) {
        float* d = reinterpret_cast<float*>(dst) + idx;
        if (RX == 4 && first == 0 && nvalid >= 4 && (idx & 3) == 0) {
            *reinterpret_cast<float4*>(d) = make_float4(v[0], v[1], v[2], v[3]);
        } else if (RX == 2 && first == 0 && nvalid >= 2 && (idx & 1) == 0) {
            *reinterpret_cast<float2*>(d) = make_float2(v[0], v[1]);
        } else {
#pragma unroll
            for (int x = 0; x < RX; ++x)
                if (x >= first && x < nvalid) d[x] = v[x];
        }
        return;
    }
    unsigned q[RX];
#pragma unroll
    for (int x = 0; x < RX; ++x) q[x] = static_cast<unsigned>(fminf(fmaxf(rintf(v[x]), 0.f), qmax));
    if (dfmt == FMT_U16) {
        uint16_t* d = reinterpret_cast<uint16_t*>(dst) + idx;
#pragma unroll
        for (int x = 0; x < RX; ++x)
            if (x >= first && x < nvalid) d[x] = static_cast<uint16_t>(q[x]);
    } else {
        unsigned char* d = reinterpret_cast<unsigned char*>(dst) + idx;
#pragma unroll
        for (int x = 0; x < RX; ++x)
            if (x >= first && x < nvalid) d[x] = static_cast<unsigned char>(q[x]);
    }
}

// ---------------------------------------------------------------------------------------
// Error-free transformations for integer destinations whose FP32 rounding error could flip
// a code: TwoProd(a, b) = (a*b, fma(a, b, -a*b)) and Knuth's TwoSum give each product and
// each addition with its rounding error exactly, accumulated as in the compensated dot
// product Dot2 (Ogita, Rump, Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput.
// 2005): a running sum s and an error sum c, whose pair (s, c) carries about twice the
// working precision.

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (s, c) += g * (h + l), with the product's rounding error recovered exactly
__device__ __forceinline__ void dot2_step(float g, float h, float l, float& s, float& c)
{
    const float p = __fmul_rn(g, h);
    float e = __fmaf_rn(g, h, -p);
    e = __fmaf_rn(g, l, e);
    float t;
    two_sum(s, p, s, t);
    c = __fadd_rn(c, __fadd_rn(t, e));
}

// (s, c) += g * h for an input h that is exact (a source code or a float32 voxel)
__device__ __forceinline__ void dot2_exact(float g, float h, float& s, float& c)
{
    const float p = __fmul_rn(g, h);
    const float e = __fmaf_rn(g, h, -p);
    float t;
    two_sum(s, p, s, t);
    c = __fadd_rn(c, __fadd_rn(t, e));
}

// (s, c) = g * (h + l) as the first term of a sum: exactly what dot2_step gives from
// s = c = 0 (TwoSum(0, p) is (p, 0)), without the addition
__device__ __forceinline__ void dot2_first(float g, float h, float l, float& s, float& c)
{
    s = __fmul_rn(g, h);
    c = __fmaf_rn(g, l, __fmaf_rn(g, h, -s));
}

// the same for an exact input h (what dot2_exact gives from s = c = 0)
__device__ __forceinline__ void dot2_first_exact(float g, float h, float& s, float& c)
{
    s = __fmul_rn(g, h);
    c = __fmaf_rn(g, h, -s);
}

// code = clamp(round-half-even(a0 + a1 * (s + c)), 0, qmax) with a0 = a0h + a0l and
// a1 = a1h + a1l double-float constants: the product and the sum are formed with their
// rounding errors, and the rounding decision is taken on the pair (u, lo)
__device__ __forceinline__ unsigned comp_code(float s, float c, float a0h, float a0l, float a1h,
                                              float a1l, float qmax)
{
    const float p = __fmul_rn(a1h, s);
    float e = __fmaf_rn(a1h, s, -p);
    e = __fmaf_rn(a1h, c, e);
    e = __fmaf_rn(a1l, s, e);
    float u, t;
    two_sum(a0h, p, u, t);
    const float lo = __fadd_rn(__fadd_rn(t, e), a0l);
    if (!(fabsf(u) < 1.0e9f)) return u > 0.f ? static_cast<unsigned>(qmax) : 0u;   // NaN -> 0
    float q = rintf(u);
    const float r = __fadd_rn(__fsub_rn(u, q), lo);   // u - q is exact
    if (r > 0.5f) q += 1.f;
    else if (r < -0.5f) q -= 1.f;
    else if (r == 0.5f || r == -0.5f) {
        const float cand = r > 0.f ? q + 1.f : q - 1.f;     // exact tie: the even code
        if (fmodf(cand, 2.f) == 0.f) q = cand;
    }
    return static_cast<unsigned>(fminf(fmaxf(q, 0.f), qmax));
}

}  // namespace vkt
