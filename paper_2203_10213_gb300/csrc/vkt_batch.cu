// vkt_batch.cu -- vktApplyFilterBatchSV: many independent (dst, src, filter) triples in one
// persistent launch over a work list of bricks, captured in a CUDA graph.
//
// Separable triples (k <= 7, any source/destination formats, any dims) become bricks of the
// fused separable pipeline (vkt_sep_brick.cuh): the host builds a per-volume table (data
// pointers, dims, formats, epilogue constants, the three weight vectors) and one TMA tensor
// map per volume whose rows allow one (others take the plain-load path), plus a work list of
// (volume, brick) items ordered by cost.  One CTA per SM slot grabs items from an atomic
// counter until the list is empty, so uneven volumes balance themselves and there is no
// per-volume launch.  Dense triples (and separable ones of k = 9, whose registers would
// slow the whole persistent kernel down) are added to the same graph as single-volume
// launches of their own path.  The graph (counter reset + persistent kernel + dense launches) is built
// once per set of handles and replayed while the same handles are passed again; the table is
// re-uploaded only when weights or value ranges changed.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <list>
#include <mutex>
#include <vector>

#include "vkt_sep_brick.cuh"

namespace vkt {
namespace {

// One persistent kernel per (filter size K, accumulation mode): its work list holds only
// bricks of volumes with that K (and, for COMP, integer destinations whose FP32 error bound
// is too loose), so its code holds one brick variant (a kernel for every K thrashed the
// instruction cache) and its registers are those of K.  The kernels of one batch run as
// parallel branches of the graph: blocks of the next kernel fill the SMs that a drained
// kernel leaves, so no kernel's tail idles the GPU.
using BatchKernel = void (*)(const sep::Job*, const CUtensorMap*, const int4*, int, unsigned*,
                             unsigned*);

template <int K, bool COMP, int BXG>
__global__ void __launch_bounds__(sep::NT, 2)
    k_sep_batch(const sep::Job* __restrict__ jobs, const CUtensorMap* __restrict__ maps,
                const int4* __restrict__ items, int nitems, unsigned* counter, unsigned* status)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int next;
    if (threadIdx.x == 0) sep::init_barriers(smem);
    __syncthreads();
    uint32_t gplane = 0;
    for (;;) {
        if (threadIdx.x == 0) next = static_cast<int>(atomicAdd(counter, 1u));
        __syncthreads();
        const int item = next;
        __syncthreads();
        if (item >= nitems) break;
        const int4 w = items[item];
        const sep::Job& J = jobs[w.x];
        const CUtensorMap* tm = maps + w.x;
        sep::W<K> G;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            G.gx[i] = J.g[0][i];
            G.gy[i] = J.g[1][i];
            G.gz[i] = J.g[2][i];
        }
        bool ok;
        if constexpr (COMP)
            ok = sep::brick_comp<K, sep::W<K>, sep::LM_ANY, false, BXG>(J, G, tm, w.y, w.z, w.w, smem,
                                                                        gplane, status);
        else
            ok = sep::brick<K, sep::W<K>, -1, -1, sep::LM_ANY, false, sep::FSTAGES, false, (K >= 5),
                            BXG>(J, G, tm, w.y, w.z, w.w, smem, gplane, status);
        if (!ok) break;
    }
}

constexpr int NKS = 4;                     // filter sizes of the persistent kernels: 1, 3, 5, 7
constexpr int KS[NKS] = {1, 3, 5, 7};
int k_slot(int k) { return k <= 1 ? 0 : (k <= 3 ? 1 : (k <= 5 ? 2 : 3)); }

// Brick shapes: the default (16 threads along x: 64 x 32 outputs, 64 x 16 compensated) and
// the narrow one for volumes it covers with less padding (8 threads along x: 32 x 32).
constexpr int BXN = 8;

template <int BXG>
BatchKernel kernel_of(int k, bool comp)
{
    switch (k) {
    case 1: return comp ? k_sep_batch<1, true, BXG> : k_sep_batch<1, false, BXG>;
    case 3: return comp ? k_sep_batch<3, true, BXG> : k_sep_batch<3, false, BXG>;
    case 5: return comp ? k_sep_batch<5, true, BXG> : k_sep_batch<5, false, BXG>;
    default: return comp ? k_sep_batch<7, true, BXG> : k_sep_batch<7, false, BXG>;
    }
}

BatchKernel batch_kernel(int k, bool comp, bool narrow)
{
    return narrow ? kernel_of<BXN>(k, comp) : kernel_of<sep::BX>(k, comp);
}

template <int BXG>
size_t smem_of(int k, int sfmt, bool comp, bool rows)
{
    if (comp) {
        switch (k) {
        case 1: return sep::smem_bytes_comp<1, BXG>(sfmt, rows);
        case 3: return sep::smem_bytes_comp<3, BXG>(sfmt, rows);
        case 5: return sep::smem_bytes_comp<5, BXG>(sfmt, rows);
        default: return sep::smem_bytes_comp<7, BXG>(sfmt, rows);
        }
    }
    switch (k) {
    case 1: return sep::smem_bytes<1, sep::FSTAGES, BXG>(sfmt, rows);
    case 3: return sep::smem_bytes<3, sep::FSTAGES, BXG>(sfmt, rows);
    case 5: return sep::smem_bytes<5, sep::FSTAGES, BXG>(sfmt, rows);
    default: return sep::smem_bytes<7, sep::FSTAGES, BXG>(sfmt, rows);
    }
}

size_t batch_smem(int k, int sfmt, bool comp, bool rows, bool narrow)
{
    return narrow ? smem_of<BXN>(k, sfmt, comp, rows) : smem_of<sep::BX>(k, sfmt, comp, rows);
}

// output tile (x, y) of a brick shape
int tile_x(bool narrow) { return narrow ? sep::tile_x<BXN>() : sep::tile_x<sep::BX>(); }
int tile_y(bool narrow, bool comp)
{
    if (comp) return narrow ? sep::tile_y_comp<BXN>() : sep::tile_y_comp<sep::BX>();
    return narrow ? sep::tile_y<BXN>() : sep::tile_y<sep::BX>();
}

// the narrow shape when it covers the volume's x-y extent with less padding
bool narrow_for(int nx, int ny, bool comp)
{
    auto area = [&](bool nw) {
        const long tx = tile_x(nw), ty = tile_y(nw, comp);
        return ((nx + tx - 1) / tx) * tx * ((ny + ty - 1) / ty) * ty;
    };
    return area(true) < area(false);
}

// TMA box width (raw voxels per stage row) of a brick with tx outputs along x
int raw_width(int tx, int sfmt) { return tx + 2 * fmt_xalign(sfmt); }

// A replayable batch: device table, tensor maps, work list, counter, and the graph.
struct Plan {
    std::vector<unsigned char> key;
    int device = -1;
    void* dmem = nullptr;
    sep::Job* d_jobs = nullptr;
    CUtensorMap* d_maps = nullptr;
    int4* d_items = nullptr;
    unsigned* d_counter = nullptr;    // one work-list counter per persistent kernel
    std::vector<sep::Job> jobs;       // table as last uploaded
    int nitems = 0;
    unsigned kernels = 0;             // kernels one replay launches
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;

    void release()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (dmem) cudaFree(dmem);
        exec = nullptr;
        graph = nullptr;
        dmem = nullptr;
    }
};

constexpr size_t MAX_PLANS = 4;
std::mutex g_plans_mutex;
std::list<Plan> g_plans;   // most recently used first

template <class T>
void put(std::vector<unsigned char>& key, const T& v)
{
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
    key.insert(key.end(), p, p + sizeof(T));
}

bool valid_volume(const vktStructuredVolume_impl* v) { return v && v->magic == VKT_VOLUME_MAGIC; }
bool valid_filter(const vktFilter_impl* f) { return f && f->magic == VKT_FILTER_MAGIC; }
int fbytes(int f) { return f == vktDataFormatUint8 ? 1 : (f == vktDataFormatUint16 ? 2 : 4); }
double fqmax(int f) { return f == vktDataFormatUint8 ? 255.0 : 65535.0; }
uint64_t vbytes(const vktStructuredVolume_impl* v)
{
    return static_cast<uint64_t>(v->dims[0]) * v->dims[1] * v->dims[2] * fbytes(v->format);
}

// The triples of a batch run at once, so a destination must be disjoint from every other
// destination and from every source of the batch (sources may be shared): a write into a
// volume that another triple reads or writes would have no defined result.  Sorting the
// destinations makes this O(n log n).
bool triples_disjoint(int n, const vktStructuredVolume* dst, const vktStructuredVolume* src)
{
    struct Span {
        uintptr_t lo, hi;
    };
    std::vector<Span> d;
    d.reserve(n);
    for (int i = 0; i < n; ++i) {
        const uintptr_t lo = reinterpret_cast<uintptr_t>(dst[i]->data);
        const uint64_t b = vbytes(dst[i]);
        if (b) d.push_back({lo, lo + b});
    }
    std::sort(d.begin(), d.end(), [](const Span& a, const Span& b) { return a.lo < b.lo; });
    for (size_t i = 1; i < d.size(); ++i)
        if (d[i].lo < d[i - 1].hi) return false;
    for (int j = 0; j < n; ++j) {
        const uintptr_t lo = reinterpret_cast<uintptr_t>(src[j]->data);
        const uint64_t b = vbytes(src[j]);
        if (!b) continue;
        const uintptr_t hi = lo + b;
        // destinations are disjoint and sorted, so their ends rise too: only the last one
        // that starts below hi can reach past lo
        auto it = std::lower_bound(d.begin(), d.end(), hi,
                                   [](const Span& s, uintptr_t v) { return s.lo < v; });
        if (it != d.begin() && (it - 1)->hi > lo) return false;
    }
    return true;
}

void epilogue_of(const vktStructuredVolume_impl* dst, const vktStructuredVolume_impl* src,
                 double wsum, float* a0, float* a1, float* qmax, float* a0lo = nullptr,
                 float* a1lo = nullptr)
{
    double ls = 0.0, ss = 1.0;
    if (src->format != vktDataFormatFloat32) {
        ls = src->lo;
        ss = (static_cast<double>(src->hi) - src->lo) / fqmax(src->format);
    }
    if (dst->format == vktDataFormatFloat32) {
        *a0 = static_cast<float>(ls * wsum);
        *a1 = static_cast<float>(ss);
        *qmax = 0.f;
    } else {
        const double sd = fqmax(dst->format) / (static_cast<double>(dst->hi) - dst->lo);
        *a0 = static_cast<float>((ls * wsum - dst->lo) * sd);
        *a1 = static_cast<float>(ss * sd);
        *qmax = static_cast<float>(fqmax(dst->format));
        if (a0lo) *a0lo = static_cast<float>((ls * wsum - dst->lo) * sd - static_cast<double>(*a0));
        if (a1lo) *a1lo = static_cast<float>(ss * sd - static_cast<double>(*a1));
    }
}

// Planes per brick along z for a volume of nz planes: whole volumes up to 1.5 x `target`
// planes, else equal chunks of about `target` planes.
int batch_zchunk(int nz, int target)
{
    if (2 * nz <= 3 * target) return nz;
    const int chunks = (nz + target - 1) / target;
    return (nz + chunks - 1) / chunks;
}

// sep_idx: triples for the persistent kernel; dense_idx: triples launched on their own
// (dense filters, and separable ones of k = 9) inside the same graph.
// zt: brick z extent target (batch_zchunk); per_sm_cap: CTAs per SM of the persistent grids
// (0: as many as the occupancy allows); narrow: volumes that the narrow brick covers with
// less padding take it
vktError build_plan(Plan& P, int32_t n, vktStructuredVolume* dst, vktStructuredVolume* src,
                    vktFilter* filters, const std::vector<int>& sep_idx,
                    const std::vector<int>& dense_idx, bool force_dense, bool force_direct,
                    const Ctx& ctx, int zt = 64, int per_sm_cap = 0, bool narrow = false)
{
    // work list: separable volumes' bricks, heavy kernels first
    std::vector<int4> items;
    size_t smem = 0;
    P.jobs.resize(sep_idx.size());
    std::vector<CUtensorMap> maps(sep_idx.size());
    std::vector<char> vnarrow(sep_idx.size(), 0);   // the brick shape of each volume
    std::vector<std::pair<long, int>> order;
    for (size_t j = 0; j < sep_idx.size(); ++j) {
        const int i = sep_idx[j];
        const vktStructuredVolume_impl* s = src[i];
        sep::Job& J = P.jobs[j];
        memset(&J, 0, sizeof(J));
        J.src = s->data;
        J.dst = dst[i]->data;
        J.nx = s->dims[0];
        J.ny = s->dims[1];
        J.nz = s->dims[2];
        sep::set_whole_volume(J);
        J.sfmt = s->format;
        J.dfmt = dst[i]->format;
        J.k = filters[i]->k;
        J.comp = separable_needs_comp(dst[i], s, filters[i]) ? 1 : 0;
        vnarrow[j] = narrow && narrow_for(J.nx, J.ny, J.comp != 0);
        const int tx = tile_x(vnarrow[j]), ty = tile_y(vnarrow[j], J.comp != 0);
        J.zchunk = batch_zchunk(J.nz, zt);
        J.tiles_x = (J.nx + tx - 1) / tx;
        J.tiles_y = (J.ny + ty - 1) / ty;
        J.chunks = (J.nz + J.zchunk - 1) / J.zchunk;
        memset(&maps[j], 0, sizeof(CUtensorMap));
        J.use_tma = encode_tensor_map_3d(&maps[j], J.sfmt, J.src, J.nx, J.ny, J.nz,
                                         raw_width(tx, J.sfmt), ty + 2 * ((J.k - 1) / 2), 1)
                        ? 1
                        : 0;
        // rows that no tensor map can describe are still fetched asynchronously, one bulk copy
        // per row, when the volume starts on a 16-byte boundary
        J.rows = (!J.use_tma && reinterpret_cast<uintptr_t>(J.src) % 16 == 0) ? 1 : 0;
        smem = std::max(smem, batch_smem(J.k, J.sfmt, J.comp != 0, J.rows != 0, vnarrow[j]));
        order.push_back({-static_cast<long>(J.k) * (J.zchunk + J.k - 1), static_cast<int>(j)});
    }
    std::stable_sort(order.begin(), order.end());
    // one work list per (K, mode), each ordered heavy bricks first
    // list l = (k slot, mode, shape): (2 * k_slot + comp) * 2 + narrow
    constexpr int NL = 4 * NKS;
    std::vector<int4> lists[NL];
    size_t lsmem[NL] = {};
    double lwork[NL] = {};
    for (const auto& o : order) {
        const sep::Job& J = P.jobs[o.second];
        const int l = (2 * k_slot(J.k) + (J.comp ? 1 : 0)) * 2 + (vnarrow[o.second] ? 1 : 0);
        lsmem[l] = std::max(lsmem[l], batch_smem(J.k, J.sfmt, J.comp != 0, J.rows != 0,
                                                 vnarrow[o.second]));
        lwork[l] += static_cast<double>(J.nx) * J.ny * J.nz * J.k * (J.comp ? 10.0 : 1.0);
        for (int bz = 0; bz < J.chunks; ++bz)
            for (int by = 0; by < J.tiles_y; ++by)
                for (int bx = 0; bx < J.tiles_x; ++bx)
                    lists[l].push_back(make_int4(o.second, bx, by, bz));
    }
    int loff[NL + 1] = {};
    for (int l = 0; l < NL; ++l) {
        loff[l + 1] = loff[l] + static_cast<int>(lists[l].size());
        items.insert(items.end(), lists[l].begin(), lists[l].end());
    }
    P.nitems = static_cast<int>(items.size());
    (void)smem;

    // one device block: table | maps (64-byte aligned) | items | one counter per list
    const size_t njobs = std::max<size_t>(1, P.jobs.size());
    const size_t off_maps = ((njobs * sizeof(sep::Job)) + 127) & ~size_t(127);
    const size_t off_items = off_maps + njobs * sizeof(CUtensorMap);
    const size_t off_counter = off_items + std::max<size_t>(1, items.size()) * sizeof(int4);
    const size_t total = off_counter + 4 * NKS * 128;   // counters 128 bytes apart
    cudaError_t e = cudaMalloc(&P.dmem, total);
    if (e != cudaSuccess) return from_cuda(e);
    unsigned char* base = static_cast<unsigned char*>(P.dmem);
    P.d_jobs = reinterpret_cast<sep::Job*>(base);
    P.d_maps = reinterpret_cast<CUtensorMap*>(base + off_maps);
    P.d_items = reinterpret_cast<int4*>(base + off_items);
    P.d_counter = reinterpret_cast<unsigned*>(base + off_counter);
    if (!P.jobs.empty()) {
        e = cudaMemcpy(P.d_jobs, P.jobs.data(), P.jobs.size() * sizeof(sep::Job), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(P.d_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !items.empty())
            e = cudaMemcpy(P.d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return from_cuda(e);
    }
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P.device);
    int lgrid[NL] = {};
    for (int l = 0; l < NL; ++l) {
        const int nl = loff[l + 1] - loff[l];
        if (nl == 0) continue;
        BatchKernel kern = batch_kernel(KS[l / 4], (l / 2) % 2 == 1, l % 2 == 1);
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(lsmem[l]));
        if (e != cudaSuccess) return from_cuda(e);
        int per_sm = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, sep::NT, lsmem[l]);
        if (per_sm_cap > 0) per_sm = std::min(per_sm, per_sm_cap);
        lgrid[l] = static_cast<int>(std::min<long>(nl, static_cast<long>(sms) * std::max(per_sm, 1)));
    }
    // lists launched heaviest first
    int lorder[NL];
    for (int l = 0; l < NL; ++l) lorder[l] = l;
    std::stable_sort(lorder, lorder + NL, [&](int a, int b) { return lwork[a] > lwork[b]; });

    // capture: counter reset, then a fork: every list's persistent kernel on a branch of its
    // own, the dense triples on the main branch, joined at the end
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return from_cuda(e);
    cudaStream_t side[NL] = {};
    cudaEvent_t fork = nullptr, join[NL] = {};
    e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int l = 0; l < NL && e == cudaSuccess; ++l) {
        if (loff[l + 1] == loff[l]) continue;
        e = cudaStreamCreateWithFlags(&side[l], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[l], cudaEventDisableTiming);
    }
    auto cleanup = [&]() {
        for (int l = 0; l < NL; ++l) {
            if (side[l]) cudaStreamDestroy(side[l]);
            if (join[l]) cudaEventDestroy(join[l]);
        }
        if (fork) cudaEventDestroy(fork);
        cudaStreamDestroy(cs);
    };
    if (e != cudaSuccess) {
        cleanup();
        return from_cuda(e);
    }
    Ctx cctx = ctx;
    cctx.stream = cs;
    uint64_t before = 0;
    vktGetLaunchCount(&before);
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    vktError err = from_cuda(e);
    unsigned kernels = 0;
    if (err == VKT_NO_ERROR && P.nitems > 0) {
        e = cudaMemsetAsync(P.d_counter, 0, NL * 128, cs);
        if (e == cudaSuccess) e = cudaEventRecord(fork, cs);
        for (int q = 0; q < NL && e == cudaSuccess; ++q) {
            const int l = lorder[q];
            const int nl = loff[l + 1] - loff[l];
            if (nl == 0) continue;
            e = cudaStreamWaitEvent(side[l], fork, 0);
            if (e != cudaSuccess) break;
            batch_kernel(KS[l / 4], (l / 2) % 2 == 1, l % 2 == 1)<<<lgrid[l], sep::NT, lsmem[l], side[l]>>>(
                P.d_jobs, P.d_maps, P.d_items + loff[l], nl, P.d_counter + 32 * l, ctx.status);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(join[l], side[l]);
            ++kernels;
        }
        err = from_cuda(e);
    }
    for (size_t q = 0; q < dense_idx.size() && err == VKT_NO_ERROR; ++q) {
        const int i = dense_idx[q];
        const vktFilter_impl* f = filters[i];
        Job job{};
        job.src = src[i]->data;
        job.dst = dst[i]->data;
        job.nx = src[i]->dims[0];
        job.ny = src[i]->dims[1];
        job.nz = src[i]->dims[2];
        job.sfmt = src[i]->format;
        job.dfmt = dst[i]->format;
        double wsum = 0.0;
        const bool sepf = f->separable && !force_dense;
        if (sepf) {
            double s3[3] = {0, 0, 0};
            for (int a = 0; a < 3; ++a)
                for (int t = 0; t < f->k; ++t) s3[a] += f->g[a][t];
            wsum = s3[0] * s3[1] * s3[2];
        } else {
            for (int t = 0; t < f->k * f->k * f->k; ++t) wsum += f->w[t];
        }
        epilogue_of(dst[i], src[i], wsum, &job.a0, &job.a1, &job.qmax, &job.a0lo, &job.a1lo);
        job.comp = (sepf ? separable_needs_comp(dst[i], src[i], f) : direct_needs_comp(dst[i], src[i], f))
                       ? 1
                       : 0;
        if (sepf)
            err = launch_separable(job, f->g[0], f->g[1], f->g[2], f->k, cctx);
        else if (f->k >= 5 && !force_direct && tensor_available(dst[i], src[i], f) == VKT_NO_ERROR)
            err = launch_tensor(job, f->w, f->k, cctx);
        else
            err = launch_direct(job, f->w, f->k, cctx);
        ++kernels;
    }
    // join the branches into the main stream before the capture ends
    for (int l = 0; l < NL && err == VKT_NO_ERROR; ++l)
        if (side[l] && loff[l + 1] > loff[l]) err = from_cuda(cudaStreamWaitEvent(cs, join[l], 0));
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    if (err == VKT_NO_ERROR) err = from_cuda(e);
    cleanup();
    uint64_t after = 0;
    vktGetLaunchCount(&after);
    uncount_launches(static_cast<unsigned>(after - before));   // captured, not launched
    if (err != VKT_NO_ERROR) {
        if (graph) cudaGraphDestroy(graph);
        return err;
    }
    P.graph = graph;
    e = cudaGraphInstantiate(&P.exec, graph, 0);
    if (e != cudaSuccess) return from_cuda(e);
    P.kernels = kernels;
    if (ctx.debug & VKT_DEBUG_LOG)
    {
        fprintf(stderr, "[vkt] batch plan: %zu separable volumes, %d bricks in %u persistent kernels,"
                " %zu single launches, brick z target %d, CTAs per SM cap %d\n", P.jobs.size(),
                P.nitems, kernels - static_cast<unsigned>(dense_idx.size()), dense_idx.size(), zt,
                per_sm_cap);
        for (int l = 0; l < NL; ++l)
            if (loff[l + 1] > loff[l])
                fprintf(stderr, "[vkt]   k=%d%s%s: %d bricks, grid %d, smem %zu\n", KS[l / 4],
                        (l / 2) % 2 ? " compensated" : "", l % 2 ? " narrow" : "",
                        loff[l + 1] - loff[l], lgrid[l], lsmem[l]);
    }
    return VKT_NO_ERROR;
}

}  // namespace
}  // namespace vkt

using namespace vkt;

extern "C" vktError vktApplyFilterBatchSV(int32_t n, vktStructuredVolume* dst, vktStructuredVolume* src,
                                          vktFilter* filters)
{
    vkt::CallRange nvtx_range("vktApplyFilterBatchSV");
    if (n < 1 || !dst || !src || !filters) return VKT_ERROR_INVALID_VALUE;
    for (int i = 0; i < n; ++i) {
        if (!valid_volume(dst[i]) || !valid_volume(src[i]) || !valid_filter(filters[i]))
            return VKT_ERROR_INVALID_HANDLE;
        for (int a = 0; a < 3; ++a)
            if (dst[i]->dims[a] != src[i]->dims[a]) return VKT_ERROR_DIMS_MISMATCH;
        const char* pd = static_cast<const char*>(dst[i]->data);
        const char* ps = static_cast<const char*>(src[i]->data);
        if (pd < ps + vbytes(src[i]) && ps < pd + vbytes(dst[i])) return VKT_ERROR_INVALID_VALUE;
    }
    if (!triples_disjoint(n, dst, src)) return VKT_ERROR_INVALID_VALUE;
    // one filter over a batch of equal volumes (a training batch): a single direct launch
    bool handled = false;
    vktError err = apply_filter_multi(n, dst, src, filters, &handled);
    if (handled) return err;
    Ctx ctx;
    err = get_context(&ctx);
    if (err != VKT_NO_ERROR) return err;
    vktExecutionPolicy pol;
    vktGetThreadExecutionPolicy(&pol);
    int dev = 0;
    cudaGetDevice(&dev);

    std::vector<int> sep_idx, dense_idx;
    std::vector<unsigned char> key;
    // the autotuner's key of the batch: its shape without the data pointers (FNV-1a hash)
    uint64_t shape_hash = 1469598103934665603ull;
    auto mix = [&](const void* v, size_t b) {
        const unsigned char* q = static_cast<const unsigned char*>(v);
        for (size_t t = 0; t < b; ++t) shape_hash = (shape_hash ^ q[t]) * 1099511628211ull;
    };
    put(key, dev);
    put(key, n);
    put(key, pol.path);
    put(key, autotune_enabled());
    for (int i = 0; i < n; ++i) {
        const bool s = filters[i]->separable && filters[i]->k <= 7 && pol.path != VKT_PATH_DIRECT &&
                       pol.path != VKT_PATH_TENSOR;
        (s ? sep_idx : dense_idx).push_back(i);
        put(key, s);
        put(key, dst[i]->data);
        put(key, src[i]->data);
        put(key, src[i]->dims);
        put(key, src[i]->format);
        put(key, dst[i]->format);
        put(key, filters[i]->k);
        put(key, s && separable_needs_comp(dst[i], src[i], filters[i]));
        const int shape[7] = {s ? 1 : 0, src[i]->dims[0], src[i]->dims[1], src[i]->dims[2],
                              static_cast<int>(src[i]->format) * 4 + static_cast<int>(dst[i]->format),
                              filters[i]->k, s && separable_needs_comp(dst[i], src[i], filters[i])};
        mix(shape, sizeof(shape));
        if (!s) {
            // dense launches bake weights and ranges into the graph
            key.insert(key.end(), reinterpret_cast<const unsigned char*>(filters[i]->w),
                       reinterpret_cast<const unsigned char*>(filters[i]->w) +
                           sizeof(float) * filters[i]->k * filters[i]->k * filters[i]->k);
            put(key, src[i]->lo);
            put(key, src[i]->hi);
            put(key, dst[i]->lo);
            put(key, dst[i]->hi);
        }
    }
    // current table contents (weights and epilogue constants of the separable volumes)
    std::vector<sep::Job> table(sep_idx.size());
    for (size_t j = 0; j < sep_idx.size(); ++j) {
        const int i = sep_idx[j];
        const vktFilter_impl* f = filters[i];
        sep::Job& J = table[j];
        memset(&J, 0, sizeof(J));
        double s3[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a)
            for (int t = 0; t < f->k; ++t) {
                J.g[a][t] = f->g[a][t];
                s3[a] += f->g[a][t];
            }
        epilogue_of(dst[i], src[i], s3[0] * s3[1] * s3[2], &J.a0, &J.a1, &J.qmax, &J.a0lo, &J.a1lo);
        J.comp = separable_needs_comp(dst[i], src[i], f) ? 1 : 0;
    }

    std::lock_guard<std::mutex> lock(g_plans_mutex);
    auto it = std::find_if(g_plans.begin(), g_plans.end(), [&](const Plan& p) { return p.key == key; });
    if (it == g_plans.end()) {
        const bool force_dense = pol.path == VKT_PATH_DIRECT || pol.path == VKT_PATH_TENSOR;
        const bool force_direct = pol.path == VKT_PATH_DIRECT;
        cudaStream_t pstream = static_cast<cudaStream_t>(pol.stream);
        // brick z extent, brick shape and persistent grid: the tuned choice of this batch
        // shape, else the rule (64-plane bricks of the default shape, as many CTAs per SM as
        // fit), else measured now.  A batch choice's `path` field holds the CTAs-per-SM cap in
        // bits 0-3 and, in bit 4, that volumes the narrow shape pads less take it (on the
        // 256-volume batch the narrow shape measured 1.31 ms against 1.27 without it: its one
        // output row per thread costs more per plane than the padding it saves).
        char tkey[96];
        std::snprintf(tkey, sizeof(tkey), "batch n%d %016llx", n,
                      static_cast<unsigned long long>(shape_hash));
        TuneChoice tc;
        tc.zchunk = 64;
        tc.path = 0;
        const bool tune = !sep_idx.empty() && autotune_enabled() && pol.path == VKT_PATH_AUTO;
        bool measure = false;
        if (tune && !autotune_lookup(tkey, &tc)) measure = !stream_capturing(pstream);
        Plan P;
        if (measure) {
            // every candidate plan is built and replayed on the policy stream; the fastest
            // is kept (the replays write the destinations, as the call itself does)
            constexpr int NC = 6;
            const TuneChoice cand[NC] = {{0, 64, 0.f},  {0, 32, 0.f},  {0, 128, 0.f},
                                         {1, 64, 0.f},  {16, 64, 0.f}, {16, 32, 0.f}};
            // (path bit 4 set: narrow bricks where they pad less; clear: the default shape)
            std::vector<Plan> plans(NC);
            for (int c = 0; c < NC && err == VKT_NO_ERROR; ++c) {
                plans[c].key = key;
                plans[c].device = dev;
                err = build_plan(plans[c], n, dst, src, filters, sep_idx, dense_idx, force_dense,
                                 force_direct, ctx, cand[c].zchunk, cand[c].path & 15,
                                 (cand[c].path & 16) != 0);
            }
            if (err == VKT_NO_ERROR) {
                err = autotune_time(cand, NC, [&](const TuneChoice& t) {
                    const int c = static_cast<int>(&t - cand);
                    count_launches(plans[c].kernels);
                    return from_cuda(cudaGraphLaunch(plans[c].exec, pstream));
                }, pstream, &tc);
            }
            int keep = -1;
            for (int c = 0; c < NC; ++c)
                if (err == VKT_NO_ERROR && cand[c].zchunk == tc.zchunk && cand[c].path == tc.path) keep = c;
            for (int c = 0; c < NC; ++c)
                if (c != keep) plans[c].release();
            if (err != VKT_NO_ERROR || keep < 0) return err != VKT_NO_ERROR ? err : VKT_ERROR_CUDA;
            autotune_store(tkey, tc);
            if (ctx.debug & VKT_DEBUG_LOG)
                fprintf(stderr, "[vkt] autotune %s: brick z target %d, CTAs per SM cap %d, "
                        "narrow bricks %s, %.4f ms\n", tkey, tc.zchunk, tc.path & 15,
                        (tc.path & 16) ? "on" : "off", tc.ms);
            P = std::move(plans[keep]);
        } else {
            P.key = key;
            P.device = dev;
            err = build_plan(P, n, dst, src, filters, sep_idx, dense_idx, force_dense, force_direct,
                             ctx, tc.zchunk > 0 ? tc.zchunk : 64, std::max(0, tc.path) & 15,
                             (std::max(0, tc.path) & 16) != 0);
            if (err != VKT_NO_ERROR) {
                P.release();
                return err;
            }
        }
        g_plans.push_front(std::move(P));
        while (g_plans.size() > MAX_PLANS) {
            g_plans.back().release();
            g_plans.pop_back();
        }
        it = g_plans.begin();
    } else if (it != g_plans.begin()) {
        g_plans.splice(g_plans.begin(), g_plans, it);
        it = g_plans.begin();
    }
    Plan& P = *it;
    cudaStream_t stream = static_cast<cudaStream_t>(pol.stream);
    // refresh weights / epilogue constants where they changed since the last upload
    for (size_t j = 0; j < table.size(); ++j) {
        sep::Job& J = P.jobs[j];
        if (memcmp(J.g, table[j].g, sizeof(J.g)) != 0 || J.a0 != table[j].a0 ||
            J.a1 != table[j].a1 || J.qmax != table[j].qmax || J.a0lo != table[j].a0lo ||
            J.a1lo != table[j].a1lo) {
            memcpy(J.g, table[j].g, sizeof(J.g));
            J.a0 = table[j].a0;
            J.a1 = table[j].a1;
            J.qmax = table[j].qmax;
            J.a0lo = table[j].a0lo;
            J.a1lo = table[j].a1lo;
            cudaError_t e = cudaMemcpyAsync(P.d_jobs + j, &J, sizeof(sep::Job),
                                            cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) return from_cuda(e);
        }
    }
    cudaError_t e = cudaGraphLaunch(P.exec, stream);
    if (e != cudaSuccess) return from_cuda(e);
    count_launches(P.kernels);
    return VKT_NO_ERROR;
}
