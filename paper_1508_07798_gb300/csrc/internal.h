// Internal declarations shared by the libhssnd translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "hssnd.h"

namespace hssnd {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define HSS_CUDA(call)                                     \
    do {                                                   \
        cudaError_t _e = (call);                           \
        if (_e != cudaSuccess) return cuda_fail(_e, #call);\
    } while (0)

#define HSS_CHECK_LAUNCH(what)                                  \
    do {                                                        \
        cudaError_t _e = cudaGetLastError();                    \
        if (_e != cudaSuccess) return cuda_fail(_e, what);      \
    } while (0)

// Raises a kernel's dynamic shared-memory limit to `bytes`, once per device
// and kernel (thread-safe); returns the runtime's error code.
cudaError_t func_smem_once(const void *func, int bytes);
int device_sms();   // multiprocessors of the current device (cached per device)

// Programmatic dependent launch.  A kernel launched by launch_pdl may begin
// while the previous kernel on its stream still runs: it calls
// pdl_launch_next() to let the kernel after it launch early, reads only what
// the previous kernel does not write, and calls pdl_wait_prev() (which returns
// once the previous kernel has completed and its writes are visible) before
// it reads or writes that kernel's output.  Launched without the attribute,
// both calls return at once.
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}
#define HSS_SMEM(kernel, bytes)                                                            \
    do {                                                                                   \
        cudaError_t _e = ::hssnd::func_smem_once((const void *)(kernel), (int)(bytes));    \
        if (_e != cudaSuccess) return cuda_fail(_e, "shared-memory attribute of " #kernel); \
    } while (0)

// Device allocation owned by a handle.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes) {
        o.p = nullptr;
        o.bytes = 0;
    }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            bytes = o.bytes;
            o.p = nullptr;
            o.bytes = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    int alloc(size_t nbytes);  // returns HSS_OK / HSS_ENOMEM
    template <class T> T *as() const { return static_cast<T *>(p); }
};

template <class T> int upload(DevBuf &b, const std::vector<T> &v, cudaStream_t s) {
    int rc = b.alloc(sizeof(T) * (v.size() ? v.size() : 1));
    if (rc) return rc;
    if (!v.empty()) HSS_CUDA(cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s));
    return HSS_OK;
}

// Scratch of one library call: a device bump allocator and a pinned host
// staging buffer for uploads.  Nothing is given back until reset() (stream
// idle: the bump pointer restarts in the first chunk) or destruction (after
// a stream synchronize), so kernels may use the memory until the next sync
// point.  Chunks and pinned buffers come from, and go back to, a
// process-wide cache (scratch_cache_*), so steady-state calls allocate
// nothing from CUDA.
struct Work {
    cudaStream_t s = nullptr;
    std::vector<DevBuf> chunks;
    size_t ci = 0;     // chunk in use
    size_t cur = 0;    // bump offset inside it
    void *hpin = nullptr;
    size_t hcap = 0, hused = 0;
    std::vector<void *> old_pins;
    std::vector<size_t> old_sizes;
    explicit Work(cudaStream_t st) : s(st) {}
    Work(const Work &) = delete;
    Work &operator=(const Work &) = delete;
    ~Work();
    int dalloc_bytes(size_t bytes, void **out);
    template <class T> int dalloc(size_t n, T **out) {
        void *p;
        int rc = dalloc_bytes(sizeof(T) * (n ? n : 1), &p);
        *out = static_cast<T *>(p);
        return rc;
    }
    int stage_bytes(const void *src, size_t bytes, void **dev);
    template <class T> int up(const std::vector<T> &v, T **out) {
        void *p;
        int rc = stage_bytes(v.data(), sizeof(T) * v.size(), &p);
        *out = static_cast<T *>(p);
        return rc;
    }
    void reset();   // the stream must be idle
    // restart the device bump pointer only: later uploads and kernels on the
    // same stream are ordered after the work that used the memory, and the
    // pinned staging keeps growing (its pending copies are not overwritten)
    void reset_device() {
        ci = 0;
        cur = 0;
    }
};

// A pointer into call scratch with the same accessor as DevBuf.
struct ScratchPtr {
    void *p = nullptr;
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Process-wide cache of scratch memory (bounded; thread-safe).
int scratch_cache_take_device(size_t min_bytes, size_t want_bytes, DevBuf &out);
void scratch_cache_give_device(DevBuf &&b);
void *scratch_cache_take_pinned(size_t min_bytes, size_t want_bytes, size_t &got);
void scratch_cache_give_pinned(void *p, size_t bytes);

// ---------------------------------------------------------------- tree
struct HssNode {          // one node of the HSS tree of a front's S (host view)
    int lo, hi;           // index range inside B^box
    int a, b;             // children (node ids inside the same front) or -1
    int depth;            // 0 = root
};

}  // namespace hssnd

struct hss_tree;
namespace hssnd {
// HSS tree over `dofs` (ascending depth-first positions) from the
// nested-dissection subtree of `box` (nd.cu); elem_positions: depth-first
// position of every element.
void hss_nodes_over(const hss_tree *t, const std::vector<int> &elem_pos, int box, const std::vector<int> &dofs,
                    std::vector<HssNode> &nodes);
std::vector<int> elem_positions(const hss_tree *t);
}  // namespace hssnd

struct hss_tree {
    int dim = 2, n[3] = {1, 1, 1}, p = 1, bs = 1, ndof = 0, nelem = 0, nbox = 0, maxlev = 0;
    hss_nd_opts opts{};
    std::vector<int> level, parent, child0, child1, lohi, pos0, pos1, ni, nb, ioff, boff;
    std::vector<int> iset, bset, fmap, perm, dfs_elem;
    std::vector<std::vector<int>> stages;  // stages[s]: boxes of level maxlev - s (deepest first)
    hssnd::DevBuf d_iset, d_bset, d_fmap;
    // HSS tree of each box's S over B^box (nodes in post-order, root last)
    std::vector<std::vector<hssnd::HssNode>> hss;
    // A forest of independent instances (nd_order_batched) concatenates the
    // instances' boxes, dofs and elements; nd_order makes a forest of one.
    int ninst = 1;
    std::vector<int> inst_top;     // first level-1 box of each instance (its sibling is inst_top + 1)
    std::vector<int> inst_dof;     // first dof of each instance, ninst + 1 entries
    std::vector<int> inst_elem;    // first element of each instance, ninst + 1 entries
    std::vector<int> box_inst;     // instance of each box
    std::vector<int> box_local;    // box id inside its instance (counter of the test matrices)
};

namespace hssnd {

// ---------------------------------------------------------------- gemm
// C = alpha * op(A) * op(B) + beta * C on a list of column-major problems.
// B == nullptr: op(B)(kk, j) is the +-1 test matrix entry of (seed, stream,
// front, row brow0 + kk, column j) (counter-based SplitMix64 sign).
// Rows [zr_lo, zr_hi) use beta = 0; columns [skip_lo, skip_hi) are not written.
template <class T> struct GemmDesc {
    const T *A;
    const T *B;
    T *C;
    int lda, ldb, ldc;
    int m, n, k;
    int transA, transB;
    T alpha, beta;
    int zr_lo, zr_hi;
    int skip_lo, skip_hi;
    uint64_t seed;
    int stream, front, brow0;
};

struct GemmTile {
    int desc;
    int tm, tn;   // tile coordinates (units of the tile size)
};

constexpr int GEMM_TM = 64;
constexpr int GEMM_TN = 64;
constexpr int GEMM_TC_TM = 128;   // tile of the tcgen05 GEMM (one MMA M x N)
constexpr int GEMM_TC_TN = 128;

template <class T>
int gemm_batched(const GemmDesc<T> *d_desc, const GemmTile *d_tiles, int ntiles, cudaStream_t s,
                 double flops = 0.0);

// Tensor-core (tcgen05, TF32) GEMM of the FP32 form: split = 1 uses the
// three-product hi/lo split (FP32 accuracy), 0 a single TF32 product.  err is
// set when a bounded wait expires.
int gemm_tc(const GemmDesc<float> *d_desc, const GemmTile *d_tiles, int ntiles, int split, int *err, cudaStream_t s,
            double flops);
void gemm_tc_tiles_for(const GemmDesc<float> &d, int desc_index, std::vector<GemmTile> &tiles);
// Sets the tensor-core kernel's shared-memory attribute on the current device
// (once per device, thread-safe) and so loads its module.
int gemm_tc_prepare();
// Tensor-core GEMM fed by TMA (tcgemm_tma.cu): the same problems and 128 x 128
// tiles as gemm_tc with the hi/lo split; for problems whose A (and B, unless
// generated) are 16-byte aligned with leading dimensions that are multiples of
// 4 floats.  gemm_tma_descs builds the tensor maps of the problems flagged in
// `use` (zero entries elsewhere) and uploads them through W.
struct TmaGemmDesc;
bool gemm_tma_eligible(const GemmDesc<float> &d);
int gemm_tma_prepare();
struct Work;
int gemm_tma_descs(const std::vector<GemmDesc<float>> &descs, const std::vector<char> &use, Work &W,
                   TmaGemmDesc **out);
// bf16: the sampling variant (generated +-1 B only): A as three BF16 terms,
// tcgen05 kind::f16 with FP32 accumulation
int gemm_tma(const TmaGemmDesc *d_descs, const GemmTile *d_tiles, int ntiles, int *err, cudaStream_t s,
             double flops, const char *prof_class = "gemm_tma", bool bf16 = false);
// C = alpha * 0 + beta * C (the product with k = 0) without descriptors.
int gemm_f32_k0(float *C, int ldc, int m, int n, float alpha, float beta, cudaStream_t s);
// Loads the module of the FP32 SIMT GEMM kernels.
int gemm_f32_prepare();

// 2 m n k of the written part of a problem
template <class T> double gemm_flops(const GemmDesc<T> &d) {
    int ncols = d.n;
    if (d.skip_hi > d.skip_lo) ncols -= std::max(0, std::min(d.n, d.skip_hi) - std::max(0, d.skip_lo));
    return 2.0 * d.m * (double)ncols * d.k;
}

template <class T>
void gemm_tiles_for(const GemmDesc<T> &d, int desc_index, std::vector<GemmTile> &tiles);

// ---------------------------------------------------------------- device helpers
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// +-1 entry (row, col) of test-matrix stream `stream` of front `front` under `seed`.
__host__ __device__ inline double rademacher(uint64_t seed, int stream, int front, int row, int col) {
    uint64_t key = seed ^ ((uint64_t)stream << 62) ^ ((uint64_t)front << 40) ^ ((uint64_t)row << 20) ^
                   (uint64_t)col;
    return (splitmix64(key) >> 63) ? -1.0 : 1.0;
}

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

}  // namespace hssnd
