/*
 * vkt.h -- C ABI of the GB300 ApplyFilter library.
 *
 * The calls follow the style of the paper's C99 interface (Sec. 3.3 and the ANSI C99
 * listing of Fig. exampleCvsCPP): opaque handles, the out-handle as first argument, a
 * "SV" suffix for the structured-volume variant of an algorithm, and a volume created
 * from its dims, data format, cell size and value range.  The paper prints only the
 * volume calls; the filter calls are this library's own, written in the same style.
 *
 * Conventions that hold for every call:
 *   - Every call returns a vktError and never throws or aborts.
 *   - All device memory is on the CUDA device that is current on the calling thread.
 *     Pointers named devPtr are device pointers; pointers named host* are host
 *     pointers (pinned memory makes the asynchronous copies truly asynchronous).
 *   - Work is enqueued on the stream of the calling thread's execution policy
 *     (vktSetThreadExecutionPolicy; the default is the legacy default stream) and the
 *     call returns without waiting.  Launch errors are returned at once; a device-side
 *     timeout of a bounded wait is recorded on the device and returned by the next
 *     vktSynchronize.
 *   - Handles are owned by the caller and released with the matching Destroy call.
 *     Destroy does not wait for work in flight: synchronise first.
 *   - Voxels are stored x fastest, then y, then z, with no row padding.
 */
#ifndef VKT_H
#define VKT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Entry points keep default visibility when the library hides everything else. */
#if defined(__GNUC__)
#define VKT_API __attribute__((visibility("default")))
#else
#define VKT_API
#endif

typedef enum vktError {
    VKT_NO_ERROR = 0,
    VKT_ERROR_INVALID_VALUE = 1,    /* bad size, format, range, NULL pointer, aliasing */
    VKT_ERROR_INVALID_HANDLE = 2,   /* NULL or already destroyed handle */
    VKT_ERROR_DIMS_MISMATCH = 3,    /* dst and src dims differ */
    VKT_ERROR_UNSUPPORTED = 4,      /* even or too large kernel, path not available */
    VKT_ERROR_OUT_OF_MEMORY = 5,
    VKT_ERROR_NO_DEVICE = 6,        /* no CUDA device or driver */
    VKT_ERROR_CUDA = 7,             /* any other CUDA runtime or driver error */
    VKT_ERROR_DEVICE_TIMEOUT = 8    /* a bounded device wait gave up (see vktSynchronize) */
} vktError;

/* Voxel storage formats (Fig. exampleCvsCPP: vktDataFormatUint8). */
typedef enum vktDataFormat {
    vktDataFormatUint8 = 0,
    vktDataFormatUint16 = 1,
    vktDataFormatFloat32 = 2
} vktDataFormat;

/* Filter evaluation paths; VKT_PATH_AUTO picks one per call from the filter and sizes. */
typedef enum vktFilterPath {
    VKT_PATH_AUTO = 0,
    VKT_PATH_DIRECT = 1,       /* FP32 CUDA-core tap loop over all k^3 taps */
    VKT_PATH_SEPARABLE = 2,    /* three fused 1-D passes; separable filters only */
    VKT_PATH_TENSOR = 3        /* FP16 hi/lo split on tcgen05 tensor cores, float32 data */
} vktFilterPath;

typedef struct vktStructuredVolume_impl* vktStructuredVolume;
typedef struct vktFilter_impl* vktFilter;

/*
 * Thread-local execution policy (Sec. 3.1: the thread-local ExecutionPolicy set and read
 * with SetThreadExecutionPolicy / GetThreadExecutionPolicy, which also switches debug
 * messages and the printing of algorithm times).  There is no device field: every call
 * runs on the current CUDA device.
 *   stream      cudaStream_t to enqueue on (NULL = legacy default stream)
 *   printTimes  nonzero: time each call with CUDA events and print it to stderr
 *               (this synchronises the stream after the call)
 *   debug       bit set of VKT_DEBUG_* flags (below)
 *   path        a vktFilterPath forcing the evaluation path (VKT_PATH_AUTO = choose)
 */
/* print path choices and launch shapes to stderr */
#define VKT_DEBUG_LOG 1
/*
 * Fault injection for tests of failure detection: every CTA of the direct path withholds
 * the TMA load of its first input plane, so its bounded wait for that plane runs out
 * (after 2 s).  The CTA then records the timeout in the device status word, waits for the
 * loads it did issue and exits without writing; the next vktSynchronize returns
 * VKT_ERROR_DEVICE_TIMEOUT and the context stays usable.  No other path reads this flag,
 * and calls whose source cannot use a tensor map (rows not 16-byte aligned) ignore it.
 */
#define VKT_DEBUG_INJECT_WAIT_TIMEOUT 2

typedef struct vktExecutionPolicy {
    void* stream;
    int32_t printTimes;
    int32_t debug;
    int32_t path;
} vktExecutionPolicy;

VKT_API vktError vktSetThreadExecutionPolicy(vktExecutionPolicy policy);
VKT_API vktError vktGetThreadExecutionPolicy(vktExecutionPolicy* policy);

/*
 * Autotuner.  Under VKT_PATH_AUTO the library picks the evaluation path and the launch shape
 * of each call (Sec. 3.2 allows a specialised implementation of an algorithm as long as its
 * behaviour stays the same; every choice here computes the same result within the method's
 * tolerance, and the brick shapes the same bits).  Without the autotuner the choice is a
 * fixed rule: separable filters take the separable path, dense k >= 5 filters on float32
 * volumes the tensor cores, the rest the direct path, with the launchers' brick z extents.
 * With it (the default; VKT_AUTOTUNE=0 in the environment starts the process with it off),
 * the first call of each call shape -- filter size and kind, formats, region or whole volume,
 * extent rounded up to powers of two per axis -- times its candidates on the policy stream
 * (the rule's path, for dense filters that the tensor path can evaluate also the other
 * path, and three brick z extents of the CUDA-core paths), keeps the fastest and uses it
 * from then on (the rule's choice unless another is more than 2 % faster).  That first call
 * synchronises the policy stream and launches each candidate eight times into the destination
 * (two interleaved passes of one untimed and three timed launches; then the chosen one once
 * more); a call made while
 * its stream is being captured into a graph uses the rule.  vktApplyFilterBatchSV tunes
 * each new batch plan the same way (brick z extent, persistent grid).  The choices live in
 * memory; when VKT_AUTOTUNE_CACHE names a file they are read from it at the first lookup and
 * written back after every new choice (JSON, see vktAutotuneSave).
 */
VKT_API vktError vktAutotuneSetEnabled(int32_t enabled);
VKT_API vktError vktAutotuneGetEnabled(int32_t* enabled);
/* Forgets every choice held in memory (a VKT_AUTOTUNE_CACHE file is not reread). */
VKT_API vktError vktAutotuneClear(void);
VKT_API vktError vktAutotuneGetCount(int32_t* count);
/* Writes the choices to `path` as {"vkt_autotune": 1, "entries": [{"key": K, "path": P,
 * "zchunk": Z, "ms": T}, ...]}, one entry per line; INVALID_VALUE if it cannot be written. */
VKT_API vktError vktAutotuneSave(const char* path);
/* Adds the entries of a file written by vktAutotuneSave; INVALID_VALUE if it cannot be read. */
VKT_API vktError vktAutotuneLoad(const char* path);

/* Short English description of an error code; never NULL. */
VKT_API const char* vktGetErrorString(vktError error);

/*
 * Waits for the policy stream and reports device-side failures recorded since the last
 * call: VKT_ERROR_DEVICE_TIMEOUT if a bounded wait inside a kernel gave up (the kernel
 * then skipped its work and its output is undefined), VKT_ERROR_CUDA on an asynchronous
 * CUDA error or when a kernel found its launch inconsistent with the tile shape it was
 * built for (it then skipped its work).  Clears the recorded device status.
 */
VKT_API vktError vktSynchronize(void);

/* Number of kernels this library has launched in this process (all threads). */
VKT_API vktError vktGetLaunchCount(uint64_t* count);

/* ------------------------------------------------------------------ structured volumes */

/*
 * Creates a structured volume (Sec. 3.2 "Volume Types"; argument order of the C99
 * listing in Fig. exampleCvsCPP: dims, format, cell size, range) owning
 * dx*dy*dz voxels of device memory on the current device, zero filled.
 *   dx,dy,dz  >= 1 voxels per axis
 *   format    storage format of one voxel
 *   sx,sy,sz  cell size (metadata, > 0)
 *   lo,hi     value range: an integer code q maps to lo + (hi-lo)*q/(2^N-1); for
 *             float32 voxels the stored value is the value and the range is metadata.
 *             Integer formats need hi != lo.
 * Errors: INVALID_VALUE (NULL out, bad dims/format/range), OUT_OF_MEMORY, NO_DEVICE.
 */
VKT_API vktError vktStructuredVolumeCreate(vktStructuredVolume* volume, int32_t dx, int32_t dy,
                                   int32_t dz, vktDataFormat format, float sx, float sy,
                                   float sz, float lo, float hi);

/*
 * Creates a non-owning view of dx*dy*dz voxels at devPtr (for instance the storage of
 * a torch tensor).  devPtr must be aligned to the voxel size and stay valid while the
 * view is used; Destroy never frees it.  Same arguments and errors as Create, plus
 * INVALID_VALUE for a NULL or misaligned devPtr, and, where a CUDA device is present, for a
 * devPtr that is neither device memory of the current device nor managed memory (host
 * memory, pinned or not, or an address no allocation covers; checked with
 * cudaPointerGetAttributes).  Without a device the pointer is recorded as given, and every
 * call that would launch a kernel on it returns NO_DEVICE.
 */
VKT_API vktError vktStructuredVolumeCreateView(vktStructuredVolume* volume, void* devPtr,
                                       int32_t dx, int32_t dy, int32_t dz,
                                       vktDataFormat format, float sx, float sy, float sz,
                                       float lo, float hi);

/* Releases the handle (and the device memory of an owning volume). */
VKT_API vktError vktStructuredVolumeDestroy(vktStructuredVolume volume);

VKT_API vktError vktStructuredVolumeGetDims(vktStructuredVolume volume, int32_t* dx, int32_t* dy,
                                    int32_t* dz);
VKT_API vktError vktStructuredVolumeGetDataFormat(vktStructuredVolume volume, vktDataFormat* format);
VKT_API vktError vktStructuredVolumeGetCellSize(vktStructuredVolume volume, float* sx, float* sy,
                                        float* sz);
VKT_API vktError vktStructuredVolumeGetVoxelMapping(vktStructuredVolume volume, float* lo, float* hi);
VKT_API vktError vktStructuredVolumeSetVoxelMapping(vktStructuredVolume volume, float lo, float hi);
/* Device pointer of the voxels and their size in bytes. */
VKT_API vktError vktStructuredVolumeGetData(vktStructuredVolume volume, void** devPtr);
VKT_API vktError vktStructuredVolumeGetSizeInBytes(vktStructuredVolume volume, uint64_t* bytes);

/* Asynchronous copies of all voxels between host memory and the volume (policy stream). */
VKT_API vktError vktStructuredVolumeSetData(vktStructuredVolume volume, const void* hostPtr);
VKT_API vktError vktStructuredVolumeCopyToHost(vktStructuredVolume volume, void* hostPtr);

/* ------------------------------------------------------------------ filters */

/* Largest supported kernel size. */
#define VKT_MAX_FILTER_SIZE 9

/*
 * Creates a dense k*k*k filter ("user-specified convolution kernel", Sec. 3.2 "Volume
 * Manipulation").  k odd, 1 <= k <= VKT_MAX_FILTER_SIZE.  hostWeights holds k^3 floats,
 * index (c*k + b)*k + a for the offsets (a-r, b-r, c-r) along (x, y, z), r = (k-1)/2;
 * NULL gives all zeros.  The filter value at voxel (x,y,z) is the clamp-to-edge
 * correlation sum_{a,b,c} w[c][b][a] * v(x+a-r, y+b-r, z+c-r).
 * Errors: INVALID_VALUE (NULL out), UNSUPPORTED (even or too large k), OUT_OF_MEMORY.
 */
VKT_API vktError vktFilterCreate(vktFilter* filter, int32_t k, const float* hostWeights);

/* Rank-1 filter w[c][b][a] = wz[c] * wy[b] * wx[a] from three k-vectors (host memory). */
VKT_API vktError vktFilterCreateSeparable(vktFilter* filter, int32_t k, const float* wx,
                                  const float* wy, const float* wz);

/*
 * Gaussian blur filter (the filter of the teaser figure and of Sec. 4.3): the sampled
 * Gaussian exp(-d^2 / (2 sigma^2)) at the integer offsets d in [-r, r], divided by its
 * sum in FP64 and stored as float32, used as the three vectors of a separable filter.
 * sigma > 0.
 */
VKT_API vktError vktFilterCreateGaussian(vktFilter* filter, int32_t k, float sigma);

/* Replaces the weights by k^3 dense weights (the filter stops being separable). */
VKT_API vktError vktFilterSetWeights(vktFilter filter, const float* hostWeights);

/*
 * Divides the weights by their sum, computed in FP64 (for a separable filter each
 * vector is divided by its own sum).  INVALID_VALUE if the sum is zero or not finite.
 */
VKT_API vktError vktFilterNormalize(vktFilter filter);

VKT_API vktError vktFilterGetSize(vktFilter filter, int32_t* k);
/* 1 if the filter is stored as three vectors, else 0. */
VKT_API vktError vktFilterIsSeparable(vktFilter filter, int32_t* separable);
/* Dense k^3 float32 weights (for a separable filter: the float32-rounded products). */
VKT_API vktError vktFilterGetWeights(vktFilter filter, float* hostWeights);
/* The three vectors of a separable filter (UNSUPPORTED for a dense one). */
VKT_API vktError vktFilterGetSeparableWeights(vktFilter filter, float* wx, float* wy, float* wz);
VKT_API vktError vktFilterDestroy(vktFilter filter);

/* ------------------------------------------------------------------ ApplyFilter */

/*
 * ApplyFilter (Sec. 3.2 "Volume Manipulation"): dst = the filter applied to src, every
 * voxel, clamp-to-edge at the faces.  Source codes are mapped through the source range
 * first; the float result is written to dst directly (float32 dst) or quantised
 * through the dst range, q = clamp(round-half-even((v-lo)/(hi-lo)*(2^N-1)), 0, 2^N-1).
 * dst and src must have equal dims (else DIMS_MISMATCH) and must not overlap in memory
 * (else INVALID_VALUE); their formats may differ.  UNSUPPORTED when the policy forces a
 * path that cannot evaluate this filter (separable path with a dense filter, tensor
 * path with a non-float32 volume or k < 3).
 */
VKT_API vktError vktApplyFilterSV(vktStructuredVolume dst, vktStructuredVolume src, vktFilter filter);

/*
 * Range version of ApplyFilter (Sec. 3.2: range algorithms operate on a region of interest
 * given as an axis-aligned box in cell coordinates; the name appends "Range").  Only the
 * dst voxels in [firstX, lastX) x [firstY, lastY) x [firstZ, lastZ) are written, with the
 * values vktApplyFilterSV would give them: the taps read the real neighbours of the region,
 * clamped at the volume's faces, not at the region's.  All other dst voxels keep their
 * contents.  The box must satisfy 0 <= first <= last <= dims on every axis (else
 * INVALID_VALUE); an empty box writes nothing.  The other rules are those of
 * vktApplyFilterSV; the tensor-core path filters whole volumes only (UNSUPPORTED when the
 * policy forces it here; VKT_PATH_AUTO uses the direct or separable path).
 */
VKT_API vktError vktApplyFilterRangeSV(vktStructuredVolume dst, vktStructuredVolume src,
                                       vktFilter filter, int32_t firstX, int32_t firstY,
                                       int32_t firstZ, int32_t lastX, int32_t lastY,
                                       int32_t lastZ);

/*
 * Batched ApplyFilter over n independent (dst[i], src[i], filters[i]) triples, with
 * the rules of vktApplyFilterSV for each triple, in one persistent launch over a
 * work list of bricks.  The launch is captured in a CUDA graph that is reused while
 * the same handles are passed again.  n >= 1.  The triples run at once: a destination
 * must not overlap another destination or any source of the batch (else INVALID_VALUE);
 * sources may be shared.
 */
VKT_API vktError vktApplyFilterBatchSV(int32_t n, vktStructuredVolume* dst, vktStructuredVolume* src,
                               vktFilter* filters);

/*
 * Gradients of y = ApplyFilter(src, filter) for float32 volumes, given gradDst = dL/dy:
 *   gradSrc     (float32 volume, dims of src, may be NULL) receives dL/dsrc, the exact
 *               adjoint of the clamp-to-edge correlation (taps that fall outside a face
 *               fold onto the face voxel);
 *   gradWeights (device float*, k^3, may be NULL) receives dL/dw[c][b][a] =
 *               sum_i gradDst[i] * src[clamp(i + (a-r, b-r, c-r))], reduced in FP64.
 * src, gradDst and gradSrc must be float32 with equal dims; gradSrc must not overlap
 * gradDst or src.
 */
VKT_API vktError vktApplyFilterBackwardSV(vktStructuredVolume gradSrc, float* gradWeights,
                                  vktStructuredVolume gradDst, vktStructuredVolume src,
                                  vktFilter filter);

/*
 * Gradients of a training batch y_b = ApplyFilter(srcs[b], filter), b = 0 .. n-1, one filter
 * for all volumes (the method's loss over a batch), given gradDsts[b] = dL/dy_b:
 *   gradSrcs    array of n float32 volumes, or NULL: gradSrcs[b] receives dL/dsrcs[b], the
 *               exact adjoint of vktApplyFilterBackwardSV;
 *   gradWeights device float*, k^3, or NULL: receives sum_b dL/dw over the whole batch, every
 *               volume's per-CTA partial sums reduced together in one FP64 pass.
 * All volumes are float32 with the dims of srcs[0] (else UNSUPPORTED / DIMS_MISMATCH); no
 * gradSrcs volume may overlap another one or any gradDsts or srcs volume (INVALID_VALUE).
 * When each array's volumes lie evenly spaced in memory (as the volumes of one batch tensor
 * do), dL/dsrc and the partial sums each take one launch over the whole batch; otherwise one
 * launch per volume, with the one reduction.  Scratch is stream ordered (cudaMallocAsync).
 */
VKT_API vktError vktApplyFilterBackwardBatchSV(int32_t n, vktStructuredVolume* gradSrcs,
                                               float* gradWeights, vktStructuredVolume* gradDsts,
                                               vktStructuredVolume* srcs, vktFilter filter);

/* ------------------------------------------------------------------ allocation-free variant */

/*
 * The paper has no counterpart to this call; it is a service for callers that cannot
 * allocate device memory.  vktApplyFilterBackwardSV takes its per-CTA partial sums from
 * stream-ordered scratch (cudaMallocAsync), and the library's first call on a device also
 * allocates a small status word.  Some hosts cannot allow that: a process whose device
 * memory is reserved up front by its own allocator (a framework's caching allocator or a
 * fixed memory budget), or latency-critical code that must avoid the allocator's locks and
 * its implicit synchronisation.  This entry point computes the same weight gradient but
 * allocates nothing: its scratch is a fixed array in the library's own device memory,
 * VKT_NOALLOC_SCRATCH_FLOATS floats (1 MiB), which every GPU that loads the library holds
 * until the process exits.
 *
 *   gradWeights  device float*, k^3 entries: dL/dw[c][b][a] = sum_i gradDst[i] *
 *                src[clamp(i + (a-r, b-r, c-r))], reduced in FP64 (as vktApplyFilterBackwardSV)
 *   gradDst, src float32 volumes with equal dims
 *
 * The first call on a device looks up the scratch array's device address (once per device,
 * with that device current); make that first call before any stream capture.  Work goes to
 * the calling thread's policy stream.  Every call on a device shares the one scratch array
 * and it keeps the previous call's contents (each call overwrites all the entries it reads),
 * so calls whose work overlaps on the GPU race: issue them on one stream, or synchronise in
 * between.  Returns VKT_ERROR_INVALID_VALUE when the volume needs more partial sums than the
 * scratch holds (one per 64 x 32 voxel column tile and z chunk, times k^3), VKT_ERROR_UNSUPPORTED
 * for non-float32 volumes, and the errors of vktApplyFilterBackwardSV otherwise.  A bounded
 * device wait that times out is recorded in a status word of this call's own (cleared at the
 * start of each call, in stream order), not in the one vktSynchronize reads; every entry of
 * gradWeights is then NaN.
 */
#define VKT_NOALLOC_SCRATCH_FLOATS (1u << 18)
VKT_API vktError vktApplyFilterWeightGradNoAllocSV(float* gradWeights, vktStructuredVolume gradDst,
                                                   vktStructuredVolume src, vktFilter filter);

/* ------------------------------------------------------------------ BrickDecompose */

/*
 * Number of bricks along each axis when `volume` is split into bricks of
 * brickX x brickY x brickZ voxels: ceil(dims / brick).  INVALID_HANDLE for a bad volume,
 * INVALID_VALUE for NULL outputs or a brick size < 1.  Needs no device.
 */
VKT_API vktError vktBrickDecomposeCountSV(int32_t* countX, int32_t* countY, int32_t* countZ,
                                          vktStructuredVolume volume, int32_t brickX,
                                          int32_t brickY, int32_t brickZ);

/*
 * BrickDecompose (Sec. 3.2, "domain decomposition algorithms": a volume split into subgrids,
 * optionally with ghost cells for interpolation).  Brick (kx, ky, kz) covers the source
 * voxels [o, o + s) with o = (kx*brickX, ky*brickY, kz*brickZ) and s = min(brick, dims - o)
 * per axis; it is written to bricks[(kz*countY + ky)*countX + kx], a volume the caller
 * created with dims s + 2*ghost and the source's format, whose voxel (i, j, k) becomes the
 * source voxel clamp(o - ghost + (i, j, k)) (stored codes copied bit for bit): ghost cells
 * inside the volume hold the neighbouring bricks' voxels, ghost cells beyond a face repeat
 * the face voxel (clamp-to-edge, the boundary rule of ApplyFilter).  numBricks must equal
 * countX*countY*countZ and ghost >= 0 (else INVALID_VALUE); a brick with the wrong dims gives
 * DIMS_MISMATCH, one with another format, or overlapping the source, INVALID_VALUE.  The
 * bricks must not overlap one another (not checked).  Asynchronous on the policy stream;
 * allocates nothing: the bricks' storage pointers are passed to the kernels as launch
 * parameters (one launch per 3968 bricks), so the caller may reuse the handle array as
 * soon as the call returns.
 */
VKT_API vktError vktBrickDecomposeSV(vktStructuredVolume* bricks, int32_t numBricks,
                                     vktStructuredVolume volume, int32_t brickX, int32_t brickY,
                                     int32_t brickZ, int32_t ghost);

/* ------------------------------------------------------------------ Render (headless) */

#define VKT_RENDER_MAX_LUT 256

/*
 * Parameters of vktRenderSV.  World coordinates are voxel units: the volume is the box
 * [0,dx] x [0,dy] x [0,dz], voxel (i,j,k) centred at (i+0.5, j+0.5, k+0.5).
 *   eye, center, up  pinhole camera at eye looking at center; up fixes the roll (must not be
 *                    parallel to center - eye)
 *   fovy             vertical field of view in radians, in (0, pi)
 *   step             sample spacing along a ray in voxel lengths, > 0
 *   termination      a ray stops once its accumulated opacity reaches this (> 1: never)
 *   background       RGBA behind the volume
 *   lutSize, lut     transfer function: lutSize (2 .. VKT_RENDER_MAX_LUT) straight RGBA
 *                    entries in host memory, entry i at normalised value i / (lutSize - 1);
 *                    alpha is the opacity of one voxel length
 */
typedef struct vktRenderParams {
    float eye[3];
    float center[3];
    float up[3];
    float fovy;
    float step;
    float termination;
    float background[4];
    int32_t lutSize;
    const float* lut;
} vktRenderParams;

/*
 * Headless Render (Sec. 3.2 "Rendering": volume ray marching with absorption and emission,
 * samples classified by an RGBA lookup table), without a window: rgba receives
 * height x width RGBA float pixels (device memory, 16-byte aligned, row 0 at the top).
 * Pixel (px, py) casts the ray through its centre,
 *   normalize(f + (2(px+0.5)/width - 1) tan(fovy/2) (width/height) r + (1 - 2(py+0.5)/height) tan(fovy/2) u),
 * f = normalize(center - eye), r = normalize(f x up), u = r x f.  The ray enters the box at
 * t0 = max(t_near, 0) and is sampled at t0 + (k + 0.5) step while inside.  A sample's value is
 * the trilinear blend of the mapped voxel values (clamped at the faces), normalised to
 * u = clamp((v - lo) / (hi - lo), 0, 1) by the volume's range and classified by the linearly
 * blended table entry; its opacity is corrected to the step, a' = 1 - (1 - a)^step, and it is
 * composited front to back (C += (1 - A) a' c, A += (1 - A) a').  The pixel is
 * (C + (1 - A) background.rgb, A + (1 - A) background.a).  INVALID_VALUE for bad parameters
 * (sizes, table, step, field of view, camera, an empty value range).  Asynchronous on the
 * policy stream; the table is copied at the call.
 */
VKT_API vktError vktRenderSV(float* rgba, int32_t width, int32_t height, vktStructuredVolume volume,
                             const vktRenderParams* params);

/* ------------------------------------------------------------------ CLAHE-3D */

/*
 * CLAHE-3D (Sec. 4.1, "Case Study: CLAHE-3D": contrast limited adaptive histogram
 * equalisation by brick decomposition, local histograms with a maximum cut-off, and linear
 * interpolation of the local results).  uint8 volumes only (else UNSUPPORTED); dst and src
 * have equal dims (else DIMS_MISMATCH) and do not overlap (else INVALID_VALUE).  The volume
 * is split into bricksX x bricksY x bricksZ bricks, which must divide the dims (else
 * INVALID_VALUE); N = voxels per brick.  Per brick: a 256-bin histogram of the codes; with
 * clipLimit > 0 every bin is cut at L = max(1, floor(clipLimit * N / 256)) and the excess E
 * is handed back, E / 256 to every bin and the remaining E mod 256 one each to bins 0,
 * step, 2 step, ... (step = max(1, 256 / (E mod 256))); clipLimit <= 0 disables the cut;
 * the brick's mapping is lut[q] = floor((255 * cdf[q] + N/2) / N).  Each voxel's code q is
 * then mapped by the trilinear blend of the 8 nearest bricks' lut[q], the voxel at brick
 * coordinate t = (x + 0.5) / s - 0.5 per axis (clamped to the brick grid), rounded half
 * to even.  Stored codes are used as they are (the value range plays no part).
 * Asynchronous on the policy stream; histograms and mappings use stream-ordered scratch.
 */
VKT_API vktError vktClahe3DSV(vktStructuredVolume dst, vktStructuredVolume src, int32_t bricksX,
                              int32_t bricksY, int32_t bricksZ, float clipLimit);

#ifdef __cplusplus
}
#endif

#endif /* VKT_H */
