/*
 * libsu3: the SU3_Bench link multiply on an NVIDIA GB300 (sm_103a), as a C ABI.
 *
 * The operation (arXiv 2103.00571, §Background "SU3_Bench"): for every site i of an L^4 lattice
 * and each of its four links j, the 3x3 complex matrix a[i].link[j] is multiplied by the fixed
 * per-direction 3x3 complex matrix b[j]:
 *     c[i].link[j].e[k][l] = sum_{m=0..2} a[i].link[j].e[k][m] * b[j].e[m][l].
 * Sites are independent; b is constant and shared by all sites (§Background, array sizes).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an su3_status; nothing throws, exits, aborts or traps on the device.
 *    A failed call leaves a message that su3_last_error() returns.
 *  - Pointers named *_dev are device (HBM) pointers owned by the caller and must be 16-byte
 *    aligned. Pointers named *_host are host pointers owned by the caller.
 *  - `stream` is a CUstream / cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Calls that take a stream only enqueue work on it and return without waiting; device-side
 *    errors surface at su3_sync().
 *  - b is always given on the host as FP64, double b[4][3][3][2] (link, row, column, re/im),
 *    and copied at call time, so the caller may free or change it as soon as the call returns.
 *  - A handle is not thread-safe: use one handle per host thread.
 */
#ifndef SU3_H
#define SU3_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SU3_ABI_VERSION 4

typedef enum {
  SU3_OK = 0,
  SU3_ERR_INVALID_ARG = 1,      /* null/misaligned pointer, bad size, stride, overlap, enum */
  SU3_ERR_UNSUPPORTED = 2,      /* a valid but unimplemented combination of forms */
  SU3_ERR_CUDA = 3,             /* a CUDA runtime call failed (message says which) */
  SU3_ERR_NOT_INITIALIZED = 4,  /* null handle */
  SU3_ERR_TIMEOUT = 5,          /* a bounded wait ran out (host deadline or device mbarrier) */
  SU3_ERR_FAULT_INJECTED = 6    /* SU3_FAULT_INJECT made this call fail on the host */
} su3_status;

/* Storage type of the real numbers. F64 computes in FP64; F32/F16/BF16 compute in FP32. */
typedef enum { SU3_F64 = 0, SU3_F32 = 1, SU3_F16 = 2, SU3_BF16 = 3 } su3_dtype;

/*
 * Representation of one link matrix. FULL18: 9 complex numbers, row major. TWOROW12: rows 0
 * and 1 only (6 complex numbers); row 2 of an SU(3) matrix is conj(row0 x row1) and is rebuilt
 * on the fly. (The paper stores all 18 reals; the two-row form is the MILC-style compression.)
 */
typedef enum { SU3_REPR_FULL18 = 0, SU3_REPR_TWOROW12 = 1 } su3_repr;

/*
 * Memory layout of an array of links. A "complex element" is (re, im) adjacent in memory.
 * Link q = 4*i + j is link j of site i; e indexes the complex elements of a link (0..8 or 0..5).
 *  AOS:     the paper's Site array (§Background, the Site structure): site i starts at byte
 *           i*site_stride_bytes, link j at +j*link_bytes, element e at +e*2*sizeof(real).
 *           Bytes of a site past its 4 links (the paper's coordinates/index/parity/pad) are
 *           never read by a kernel as data and never written. With a stride wider than the links
 *           the array moves through 2-D tensor copies (rows = sites) and may hold at most
 *           2^31 - 1 sites (SU3_ERR_INVALID_ARG beyond).
 *  AOSOA32: blocks of 32 links; element e of link q at complex index
 *           ((q/32)*n_elem + e)*32 + q%32. The last block is padded to 32 links.
 *  SOA:     element e of link q at complex index e*n_links + q.
 */
typedef enum { SU3_LAYOUT_AOS = 0, SU3_LAYOUT_AOSOA32 = 1, SU3_LAYOUT_SOA = 2 } su3_layout;

/*
 * Arithmetic of the F64 storage type. NATIVE: FP64 fused multiply-adds (the plain method).
 * F32PAIR: FP64 storage, arithmetic on unevaluated pairs of FP32 numbers. Each a element is split
 * into hi + lo with integer operations; each output real is a compensated dot product (TwoSum on
 * the running FP32 sum, the product error and the product's share of the TwoSum error added by one
 * FMA, error terms accumulated in a second FP32 number) and becomes FP64 with one FP64 add.
 * GB300's FP64 units run at 1/64 of its FP32 rate, so this is several times faster. Accuracy: about 2^-45 times
 * sum_m |a[k][m]||b[m][l]| per output (measured max 3.3e-14 against the FP64 oracle on SU(3)
 * data, whose entries are <= 1). Valid for finite inputs with |x| < 2^127; input magnitudes below
 * 2^-74 (including zeros) act as values below 2^-73. All repr pairs are supported; for
 * TWOROW12 -> FULL18, row 2 of a is rebuilt as conj(row0 x row1) in FP32-pair arithmetic too
 * (each real a 4-term compensated dot product of the pair splits of rows 0 and 1).
 * Must be NATIVE for F32/F16/BF16 storage (HYBRID, below, likewise).
 * Batched F64 items may use NATIVE or F32PAIR.
 */
typedef enum { SU3_ARITH_NATIVE = 0, SU3_ARITH_F32PAIR = 1, SU3_ARITH_HYBRID = 2 } su3_arith;
/*
 * SU3_ARITH_HYBRID (F64 storage): in every CTA the first round(native_permille/1000 * warps) warps
 * compute their links with NATIVE FP64 FMAs on the FP64 pipe while the other warps use F32PAIR on
 * the FP32 pipe, so both pipes work at once. Each link's result is exactly what NATIVE or F32PAIR
 * would produce for it; accuracy is that of F32PAIR. Same repr and range rules as F32PAIR.
 */

typedef struct {
  int32_t dtype;              /* su3_dtype */
  int32_t repr;               /* su3_repr */
  int32_t layout;             /* su3_layout */
  int32_t arith;              /* su3_arith */
  int64_t n_sites;            /* number of sites (4 links each); 0 is a valid no-op */
  int64_t site_stride_bytes;  /* AOS only: bytes between sites; 0 = packed (4*link bytes);
                                 otherwise >= 4*link bytes and a multiple of 16 */
} su3_desc;

typedef struct su3_handle su3_handle;

/* Launch configuration of the streaming kernels (for the autotuner); 0 fields = default.
 * AOS always streams through shared memory (the staged kernel). AOSOA32 and SOA use the staged
 * kernel when stages is 2..8 and plain coalesced global loads when stages is 0 (their default). */
typedef struct {
  int32_t block;        /* threads per CTA: a multiple of 32 in [32, 256] */
  int32_t tile_sites;   /* staged: sites per shared-memory tile (1..1024, at most 1 MiB; AOSOA32 a
                           multiple of 8, SOA at most 64; AOS/AOSOA32 tiles are shrunk at launch
                           until ctas_per_sm CTAs fit in one SM's shared memory, and AOS tiles of
                           padded sites to at most 256, the rows of one tensor copy);
                           AOSOA32/SOA direct loads: links per thread (1, 2 or 4) */
  int32_t stages;       /* staged: shared-memory pipeline depth (2..8); AOSOA32/SOA: 0 = direct */
  int32_t ctas_per_sm;  /* CTAs per SM in the persistent grid (1..32) */
  int32_t native_permille;  /* HYBRID only: share of each CTA's warps computing natively, 1/1000 */
  int32_t threads_per_link; /* staged: 1 = one thread computes a whole link (default); 3 = one
                               thread per output row (row split: three threads per link, two for
                               TWOROW12 output). su3_mult_op SU3_OP_AN and su3_mat_vec always use 1.
                               Direct loads: 1. su3_set_batched_cfg: 1 or 3. */
} su3_launch_cfg;

/* One lattice of a batched call. a/c are device pointers; b as in su3_mult. */
typedef struct {
  su3_desc desc;     /* dtype F64 or F32, FULL18, AOS packed; arith NATIVE, or F32PAIR for F64 */
  const void* a_dev;
  void* c_dev;
  double b[4][3][3][2];
} su3_batch_item;

/* ---- lifetime ---------------------------------------------------------------------------- */

/* Binds a new handle to CUDA device `device`. The handle owns a small status word in device
 * memory and the batched workspace. Every call on the handle runs on the handle's device,
 * whichever device is current, and leaves the calling thread's current device as it was
 * (su3_init too); the pointers and streams passed in must belong to the handle's device. A handle
 * is not thread-safe: use one per host thread. */
su3_status su3_init(int device, su3_handle** out);

/* Releases everything the handle owns (after synchronising its device). NULL is a no-op. */
su3_status su3_finalize(su3_handle* h);

/* ---- the operation ----------------------------------------------------------------------- */

/*
 * c = a x b[j] for every link (the SU3_Bench kernel, §Background). `a_desc` describes a_dev and
 * `c_desc` describes c_dev (NULL = same as a_desc). Both must have the same dtype, layout,
 * arith and n_sites. Supported repr pairs (a -> c): FULL18 -> FULL18, TWOROW12 -> TWOROW12
 * (rows 0-1 of c only), TWOROW12 -> FULL18 (row 2 of a rebuilt in registers).
 * a_dev == c_dev (exactly in place, same desc) is allowed; any other overlap is INVALID_ARG.
 * For F16/BF16/F32 storage, b is rounded once to FP32; results are rounded once to storage.
 * Asynchronous on `stream`: the call only enqueues work there (b travels by value in the launch
 * parameters), so it can be captured into a CUDA graph on a capturing stream and replayed, with the
 * eager call's bits (tested); make one eager call of the same form first, outside the capture.
 */
su3_status su3_mult(su3_handle* h, const su3_desc* a_desc, const void* a_dev,
                    const double* b, const su3_desc* c_desc, void* c_dev, void* stream);

/*
 * The adjacent SU(3) products (the paper's introduction places SU(3) products with matrices and
 * with colour vectors at the core of lattice-QCD codes such as MILC), with b fixed per link
 * direction as in su3_mult:
 *   SU3_OP_NN: c = a x b           (exactly su3_mult)
 *   SU3_OP_NA: c = a x b^dagger    (b^dagger formed exactly on the host, then the su3_mult path;
 *                                    every form su3_mult supports)
 *   SU3_OP_AN: c = a^dagger x b    (its own kernel: AOS, FULL18 -> FULL18, NATIVE for any dtype
 *                                    or F32PAIR for F64)
 * Same conventions as su3_mult (asynchronous, caller-owned 16-byte-aligned device buffers).
 */
typedef enum { SU3_OP_NN = 0, SU3_OP_NA = 1, SU3_OP_AN = 2 } su3_op;
su3_status su3_mult_op(su3_handle* h, int32_t op, const su3_desc* a_desc, const void* a_dev,
                       const double* b, const su3_desc* c_desc, void* c_dev, void* stream);

/*
 * Matrix x colour vector (MILC's mult_su3_mat_vec; with adjoint != 0 its adjoint form):
 *   w[i][j][k] = sum_m a[i][j][k][m] v[j][m]        or   sum_m conj(a[i][j][m][k]) v[j][m].
 * a: AOS FULL18 array of any dtype, NATIVE arithmetic (or F32PAIR for F64; packed or strided
 * sites); v: host FP64
 * double v[4][3][2], one colour vector per link direction, copied at call time (rounded once to
 * FP32 for F32/F16/BF16 storage); w_dev: packed array of n_sites x 4 colour vectors (3 complex
 * each) in a's dtype, n_sites * 12 * 2 * sizeof(real) bytes, caller-owned, not overlapping a.
 * Asynchronous on `stream`.
 */
su3_status su3_mat_vec(su3_handle* h, int32_t adjoint, const su3_desc* a_desc, const void* a_dev,
                       const double* v, void* w_dev, void* stream);

/*
 * The same operation with HOST buffers: returns when c_host is complete (synchronous). Two paths:
 *  - DIRECT: when a_host and c_host each lie inside one pinned, mapped host allocation
 *    (cudaMallocHost, cudaHostAlloc, cudaHostRegister), the kernel itself streams a in and c out
 *    over the host link (NVLink-C2C on GB300), with coalesced 16-byte loads and stores from the
 *    SMs and no staging buffer; nothing is allocated. Both ends of each range are checked; a
 *    range that spans several allocations must not be passed. On a device that reads pageable
 *    host memory coherently (su3_host_pageable_access() == 1: the GPU translates host addresses
 *    through the host's page tables, as on GB300 over NVLink-C2C), ordinary pageable memory
 *    (malloc, numpy) qualifies too: the kernel reads and writes it as it stands. Pages that the
 *    host never touched are first populated by the operating system, slowly, on either path.
 *    The kernel moves 16-byte words, so both buffers must be 16-byte aligned for this path.
 *  - STAGED: otherwise (pageable memory on other devices), a_host is copied to the device in
 *    chunks, multiplied and copied back into c_host, copies and kernels overlapped on the
 *    handle's streams. This allocates device staging buffers owned by the handle (three buffers
 *    of ~64 MB of input each) on the first call and whenever a larger site stride needs more;
 *    growing them synchronises the device before freeing the old ones.
 * su3_set_host_path chooses between them; su3_last_host_path reports which one the last call took.
 * AOS layout only. Any arith, repr pair and site stride that su3_mult supports.
 */
su3_status su3_mult_host(su3_handle* h, const su3_desc* a_desc, const void* a_host,
                         const double* b, const su3_desc* c_desc, void* c_host, void* stream);

/* Path of su3_mult_host: AUTO (default) takes DIRECT when both buffers qualify (pinned and
 * mapped, or pageable on a device with coherent pageable access), else STAGED; DIRECT fails with
 * SU3_ERR_INVALID_ARG when they do not; STAGED always copies through HBM. */
typedef enum { SU3_HOST_AUTO = 0, SU3_HOST_DIRECT = 1, SU3_HOST_STAGED = 2 } su3_host_path;
su3_status su3_set_host_path(su3_handle* h, int32_t path);
/* SU3_HOST_DIRECT or SU3_HOST_STAGED: the path of the handle's last su3_mult_host call (0: none). */
int32_t su3_last_host_path(const su3_handle* h);
/* 1 when the handle's device reads and writes pageable host memory coherently
 * (cudaDevAttrPageableMemoryAccess), so that the direct host path also takes pageable buffers;
 * 0 otherwise or for a null handle. */
int32_t su3_host_pageable_access(const su3_handle* h);

/*
 * Many independent lattices (each its own a, b, c, n_sites and storage type) in ONE persistent
 * kernel launch: the link tiles of all lattices form one global work list that the CTAs
 * stride over. With use_graph != 0 the launch (descriptor upload + kernel) is captured once into
 * a CUDA graph keyed by the item list and replayed with cudaGraphLaunch on later identical calls.
 * Supported items: dtype F64 or F32, FULL18, AOS packed; NATIVE arithmetic, or F32PAIR for F64
 * items (b is split into FP32 pairs on the host). The item array is copied at
 * call time into handle-owned device memory (the handle's workspace). Without a graph that
 * workspace is reused by every call: a call's upload is ordered on the GPU after the previous
 * call's kernel (an event wait), so calls from one handle may use different streams.
 */
su3_status su3_mult_batched(su3_handle* h, int32_t n, const su3_batch_item* items, void* stream,
                            int32_t use_graph);

/* Largest number of non-empty lattices one su3_mult_batched_static call accepts. */
#define SU3_STATIC_MAX_LATTICES 256

/*
 * su3_mult_batched for callers that cannot allocate device memory. (The paper has no
 * counterpart: this is a deployment convenience.) Some callers may not call cudaMalloc or
 * cudaFree at all: plug-ins whose host application owns every device allocation through its own
 * pool or fixed memory budget, and loops that must never stall, since cudaMalloc/cudaFree can
 * synchronise the whole device. Those callers cannot create a handle either (su3_init allocates),
 * so this entry point takes none and allocates nothing: the lattice descriptors go into a
 * statically allocated device area of 256 + SU3_STATIC_MAX_LATTICES * 1192 bytes (about 298 KB),
 * which every GPU that loads libsu3 holds until the process exits.
 *  - Runs on the calling thread's current CUDA device. The first call on each device looks up the
 *    area's device address (set-up, once per device); make that first call before any stream
 *    capture.
 *  - Items follow su3_mult_batched's rules (F64 or F32, FULL18, packed AOS, NATIVE or F64
 *    F32PAIR; a_dev/c_dev caller-owned device buffers). More than SU3_STATIC_MAX_LATTICES
 *    non-empty items returns SU3_ERR_INVALID_ARG before anything is enqueued.
 *  - Synchronous: enqueues the descriptor upload and one kernel on `stream`, waits for `stream`,
 *    and returns SU3_ERR_TIMEOUT if a device-side bounded wait ran out (the status word at the
 *    start of the area, cleared at every call), SU3_ERR_CUDA on a CUDA error.
 *  - Every call on a device shares the one area, which keeps the last call's descriptors (the
 *    status word is cleared at each call). Two calls whose work overlapped on the GPU would race
 *    on it, so the library runs one call at a time per process: a lock is held from the
 *    descriptor upload until the call's stream has drained. The descriptors are built in a
 *    static host table of SU3_STATIC_MAX_LATTICES entries and uploaded with one copy.
 */
su3_status su3_mult_batched_static(int32_t n, const su3_batch_item* items, void* stream);

/* ---- layout and precision conversion (outside the timed path) --------------------------- */

/*
 * Converts packed FP64 AOS sites (72 doubles each, the benchmark's input format) into the form
 * `dst` describes: each real rounded once, to nearest even, straight from FP64; TWOROW12 drops
 * row 2. dst->n_sites sites are converted.
 */
su3_status su3_pack(su3_handle* h, const double* aos_f64_dev, const su3_desc* dst, void* dst_dev,
                    void* stream);

/*
 * Converts an array in the form `src` describes back to packed FP64 AOS sites (exact widening;
 * TWOROW12 gets row 2 rebuilt as conj(row0 x row1) in FP64).
 */
su3_status su3_unpack(su3_handle* h, const su3_desc* src, const void* src_dev, double* aos_f64_dev,
                      void* stream);

/* ---- completion, errors, sizes, tuning --------------------------------------------------- */

/*
 * Waits for all work enqueued on `stream` (timeout_ms < 0: no host deadline; otherwise polls
 * until the deadline and returns SU3_ERR_TIMEOUT if the work is still running). Then reads and
 * clears the handle's device status word: a device-side bounded wait that ran out is reported
 * as SU3_ERR_TIMEOUT, an asynchronous CUDA error as SU3_ERR_CUDA.
 */
su3_status su3_sync(su3_handle* h, void* stream, int32_t timeout_ms);

const char* su3_status_string(su3_status s);
const char* su3_last_error(const su3_handle* h);

/* Bytes of one link (18 or 12 reals of the dtype) and bytes an array of `d` occupies. */
int64_t su3_link_bytes(int32_t dtype, int32_t repr);
int64_t su3_array_bytes(const su3_desc* d);

/* Validates a descriptor without touching the GPU (returns INVALID_ARG/UNSUPPORTED/OK). */
su3_status su3_check_desc(const su3_desc* d);

/* Per-form launch configuration used by su3_mult (the autotuner writes it), for `form` as both a
 * and c (same repr). su3_get_launch_cfg reports the configuration in force (the default if none
 * was set). */
su3_status su3_set_launch_cfg(su3_handle* h, const su3_desc* form, const su3_launch_cfg* cfg);
su3_status su3_get_launch_cfg(su3_handle* h, const su3_desc* form, su3_launch_cfg* cfg);
/* The same for one (a, c) repr pair: only c_form's repr is read. TWOROW12 -> FULL18 may take a
 * launch shape of its own; without one it uses the TWOROW12 -> TWOROW12 configuration. */
su3_status su3_set_launch_cfg_for(su3_handle* h, const su3_desc* a_form, const su3_desc* c_form,
                                  const su3_launch_cfg* cfg);
su3_status su3_get_launch_cfg_for(su3_handle* h, const su3_desc* a_form, const su3_desc* c_form,
                                  su3_launch_cfg* cfg);

/* Launch configuration of su3_mult_batched. A work tile is tile_sites * 576 bytes of input:
 * tile_sites sites of an F64 lattice or 2 * tile_sites sites of an F32 lattice. The cached graph
 * is rebuilt on the next graph-mode call. 0 fields keep the current value. */
su3_status su3_set_batched_cfg(su3_handle* h, const su3_launch_cfg* cfg);
su3_status su3_get_batched_cfg(su3_handle* h, su3_launch_cfg* cfg);

/* Number of kernel launches this handle has made since su3_init (for launch accounting). */
int64_t su3_launch_count(const su3_handle* h);

/*
 * Failure-path self test (not part of the operation): launches one CTA that waits, through the
 * same bounded mbarrier wait every streaming kernel uses, on a barrier that nothing completes,
 * with a limit of `limit_ms` (1..2000) instead of the kernels' 4 s. The kernel then records a
 * timeout in the handle's status word and returns, so a following su3_sync() must report
 * SU3_ERR_TIMEOUT while the CUDA context stays usable.
 */
su3_status su3_selftest_wait_timeout(su3_handle* h, int32_t limit_ms, void* stream);

/*
 * Diagnostic (not part of the operation): the device's sustained FP64 fused multiply-add rate in
 * TFLOP/s (2 flop per FMA), measured with 2,048 threads per SM each running 8 independent FMA
 * chains of `steps` FMAs (1..2^24; ~8192 takes tens of milliseconds on GB300). It is the
 * measured peak of the FP64 pipe that bounds the plain FP64 kernel. Synchronous; allocates a
 * small scratch buffer for the duration of the call.
 */
su3_status su3_measure_fp64_rate(su3_handle* h, int32_t steps, double* tflops);

int32_t su3_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SU3_H */
