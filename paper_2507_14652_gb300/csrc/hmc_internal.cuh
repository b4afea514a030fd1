// hmc_internal.cuh -- structures shared by the translation units of libhmc.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <memory>
#include <utility>
#include <string>
#include <vector>

#include "hmc.h"

namespace hmc {

constexpr int MAXL = HMC_MAX_LAYERS;
constexpr int MAX_SCATTER_BUFS = 40;

// Thread-local error message behind hmc_last_error().
void set_error(const char *fmt, ...);

// Status helpers: every CUDA call on the host goes through CK().
struct Fail {
    hmc_status st;
};
#define HMC_CK(call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            ::hmc::set_error("%s failed at %s:%d: %s", #call, __FILE__, __LINE__,       \
                             cudaGetErrorString(e_));                                  \
            throw ::hmc::Fail{e_ == cudaErrorMemoryAllocation ? HMC_ERR_OOM : HMC_ERR_CUDA}; \
        }                                                                              \
    } while (0)
#define HMC_LAUNCH_CK() HMC_CK(cudaGetLastError())
#define HMC_REQUIRE(cond, ...)                                                         \
    do {                                                                               \
        if (!(cond)) {                                                                 \
            ::hmc::set_error(__VA_ARGS__);                                             \
            throw ::hmc::Fail{HMC_ERR_ARG};                                            \
        }                                                                              \
    } while (0)

// One feed-forward stack with its parameter offsets inside the problem's theta.
struct NetDesc {
    int L = 0;
    int w[MAXL + 1] = {};
    int act[MAXL] = {};
    int bias[MAXL] = {};
    long woff[MAXL] = {};
    long boff[MAXL] = {};   // -1 when the layer has no bias
    long base = 0;          // offset of the first parameter of this net
    long P = 0;             // parameters of this net
    int lmin = 0;           // lowest layer that holds a sampled parameter
    bool any_sampled = false;
};

// Where the drift kernel writes each sampled coordinate (one plan per problem).
struct ScatterPlan {
    int nbuf = 0;
    void *base[MAX_SCATTER_BUFS] = {};
    long cstride[MAX_SCATTER_BUFS] = {};   // elements between chains
    int kind16[MAX_SCATTER_BUFS] = {};     // element type: 0 float, 1 bf16, 2 fp16
    void *base_lo[MAX_SCATTER_BUFS] = {};  // 16-bit buffers only: receives h16(q - hi) when set
    const uint8_t *buf_id = nullptr;       // [k] (nullptr: all in buffer 0)
    const int *off = nullptr;              // [k] element offset inside one chain's slice
};

// Per-(problem) view used by the trajectory kernels; lives in device memory.
struct SegDesc {
    long qoff;     // offset of this problem's [C][k] block in the packed state
    int k;
    int problem;   // Philox stream of this problem
    ScatterPlan sc;
};

struct Problem;
struct RowArena;

// Engine interface: U and grad U of one problem for all its chains.
struct Engine {
    virtual ~Engine() {}
    // q, g: [C][k] device, handle precision. U: [C] device doubles.
    // The sampled coordinates are assumed already scattered into the network
    // when `scattered` is true (the trajectory kernels do it in the drift).
    virtual void energy_grad(const void *q, double *U, void *g, bool scattered, cudaStream_t s) = 0;
    // Write q [C][k] into the engine's parameter buffers (what energy_grad does first
    // when `scattered` is false).
    virtual void scatter(const void *q, cudaStream_t s) = 0;
    virtual ScatterPlan scatter_plan() = 0;
    virtual size_t bytes() const = 0;
    // The energy for the Metropolis test.  Engines whose energy_grad U is only as
    // accurate as their reduced-precision gradient (the bf16 tensor-core engines)
    // provide a second, accurate U(q); q is already scattered into the network.
    virtual bool has_accurate_energy() const { return false; }
    virtual void accurate_energy(const void *q, double *U, cudaStream_t s) {}
    // what the engine's autotuner chose at creation ("" if it tunes nothing)
    virtual std::string tuning() const { return std::string(); }
    // device flag its kernels raise when a bounded wait gives up (nullptr: no such waits)
    virtual int *error_flag() const { return nullptr; }
};

// Several problems' gradients as grouped launches: one launch per kernel and layer slot
// for all of them instead of one per problem.  Built by an engine family from its own
// engines (make_umma_groups_*); each problem keeps its buffers, maps and tuning.
struct EngineGroup {
    virtual ~EngineGroup() {}
    // q, g: a batch handle's packed [problem][chain][k_problem] arrays; U: [problem][C].
    // Only the group's problems are written.
    virtual void energy_grad(const void *q, double *U, void *g, bool scattered, cudaStream_t s) = 0;
    virtual std::string describe() const = 0;
};

struct Problem {
    int kind = 0;
    NetDesc net, branch, trunk;
    int out_bias = 0;
    long b0_off = -1;
    long P = 0, k = 0;
    int C = 0;
    long n = 0;
    int dx = 0, dout = 0;
    long n_u = 0, n_y = 0;
    int du = 0, dy = 0;
    double sigma = 1.0, alpha = 1.0;
    std::vector<long> idx;          // host copy, ascending
    std::vector<double> frozen;     // host copy
    std::vector<double> x, y, u, yq, t;   // host copies of the data (FP64)
    Engine *engine = nullptr;
    RowArena *arena = nullptr;      // set for the chunk engines of a chunked handle
    bool batch_member = false;      // one of several problems of a batch handle
};

void build_net_desc(NetDesc &nd, const hmc_mlp_spec &s, long base, const std::vector<long> &idx);

// Engines (one per precision family).
Engine *make_simt_engine_f64(Problem &p, int C);
Engine *make_simt_engine_f32(Problem &p, int C);
Engine *make_umma_engine_bf16(Problem &p, int C);
Engine *make_umma_engine_f16(Problem &p, int C);
bool umma_engine_supports(const Problem &p, std::string *why);
Engine *make_don_engine_bf16(Problem &p, int C);
Engine *make_don_engine_f16(Problem &p, int C);
// Groups of the tensor-core MLP engines in `es` that share a kernel shape (padded width,
// input width, kernel family), two or more problems each; problem i's coordinates start
// at element qoff[i] of the packed q, its energies at uoff[i] of U.  Sets grouped[i]
// for every problem placed in a group.
std::vector<std::unique_ptr<EngineGroup>> make_umma_groups_bf16(const std::vector<Engine *> &es,
                                                                const std::vector<long> &qoff,
                                                                const std::vector<long> &uoff, std::vector<bool> &grouped);
std::vector<std::unique_ptr<EngineGroup>> make_umma_groups_f16(const std::vector<Engine *> &es,
                                                               const std::vector<long> &qoff,
                                                               const std::vector<long> &uoff, std::vector<bool> &grouped);
// One bounded device-side wait run out on purpose; it raises *err (hmc_diag_expire_wait).
void expire_wait_run(int *err, long limit_ns, cudaStream_t s);

// A problem without data terms: U = |q|^2 / (2 alpha^2) in any precision.
Engine *make_prior_engine(const Problem &p, int prec, int C);
bool don_engine_supports(const Problem &p, std::string *why);

// Sensitivities and truncation (k_sens.cu): a network and its inputs, no subset.
struct SensProblem {
    int kind = 0;
    NetDesc net, branch, trunk;
    int out_bias = 0;
    long P = 0;
    long n = 0, n_u = 0, n_y = 0;
    std::vector<double> x, u, yq;   // host copies of the inputs (FP64)
};
// S2 [P] (device) from the VI means mu and standard deviations sd [P] (device).
void sensitivity_run(const SensProblem &pr, int prec, const double *mu, const double *sd, double *S2,
                     cudaStream_t s);
// mask [P] (device) and the ranking order [P] (device, may be null) from S2 (device); returns N-hat.
long select_subset_run(const double *S2, long P, double tau, unsigned char *mask, long long *order,
                       cudaStream_t s);

// Posterior predictive (k_predict.cu): a problem's network, frozen vector and subset,
// with new inputs (and, for the error, their targets).
struct PredictInput {
    int kind = 0;
    NetDesc net, branch, trunk;
    int out_bias = 0;
    long P = 0;
    std::vector<double> frozen;
    std::vector<long> idx;
    long n = 0, n_u = 0, n_y = 0;
    std::vector<double> x, u, yq, targets;   // host copies (FP64)
};
// mean, sd [outputs] (device) over S samples [S][k] (device, handle precision); rel_l2
// (host, may be null) the mean relative L2 error of the mean against the targets.
void predict_run(const PredictInput &in, int prec, const void *samples, long S, double *mean, double *sd,
                 double *rel_l2, cudaStream_t s);

// Programmatic dependent launch.  A kernel started with launch_pdl may begin while
// the previous kernel in its stream drains: it runs pdl_wait() before it touches any
// global memory (that returns once the previous grid has finished and its writes are
// visible), and pdl_trigger() lets the next kernel start its own prologue early.
// Every kernel launched this way calls pdl_wait() in every block, so the completion
// of any kernel implies the completion of all kernels before it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args)
{
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
    HMC_CK(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
}

// Per-kernel timing for hmc_diag_profile_energy_grad: while a profiler is active on
// this thread, every launch site records a CUDA event pair on its launching stream.
struct Profiler {
    struct Rec {
        const char *name;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
};
Profiler *&active_profiler();
struct ProfScope {
    Profiler *p;
    cudaStream_t s;
    size_t i = 0;
    ProfScope(const char *name, cudaStream_t st);
    ~ProfScope();
};

// Device allocation helper that tracks bytes and frees on destruction.  A view
// (own = false) refers to memory another DevBuf owns and frees nothing.
struct DevBuf {
    void *ptr = nullptr;
    size_t n = 0;
    bool own = true;
    DevBuf() {}
    explicit DevBuf(size_t bytes) { alloc(bytes); }
    void alloc(size_t bytes);
    void view(void *p, size_t bytes);
    ~DevBuf();
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    template <typename T> T *as() const { return reinterpret_cast<T *>(ptr); }
};

// Device memory shared by the chunk engines of one handle (hmc_create_chunked).  They
// evaluate their rows one after another on one stream, so every buffer whose size grows
// with the rows (activations, deltas, operator outputs, split-K partials) is in use by one
// engine at a time.  An engine's k-th request gets slot k; the engines are created
// largest chunk first, so the first request of a slot fixes its size.
struct RowArena {
    std::vector<std::unique_ptr<DevBuf>> slots;
    size_t next = 0;
    void begin() { next = 0; }
    // a view of the next slot, at least `bytes` long
    void take(DevBuf &dst, size_t bytes);
    size_t bytes() const
    {
        size_t b = 0;
        for (auto &s : slots) b += s->n;
        return b;
    }
};

// A buffer that scales with the data rows: a view into the arena when the engine belongs
// to a chunked handle, else memory of its own.
inline void row_alloc(RowArena *arena, DevBuf &dst, size_t bytes)
{
    if (arena) arena->take(dst, bytes);
    else dst.alloc(bytes);
}

}  // namespace hmc
