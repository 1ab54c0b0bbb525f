// handle.h -- the library handle (workspace, saved factors, events) and
// small host helpers shared by the C-ABI translation units.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "internal.h"
#include "sqrtm_mp.h"
#include "sqrtm_mp_steps.h"

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
constexpr int kBatchPhases = 5;

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct sqrtm_handle_s {
    cudaStream_t stream = nullptr;
    Buf ws;        // scratch, reused by every call
    Buf fact;      // saved low-precision factors (Q, S or V, lam) of the last forward call
    Buf staging;   // pinned host scalars
    int64_t fact_n = -1;          // size of the saved factors, -1 = none
    void *fact_q = nullptr;       // general: Q (c64); SPD: V (float)
    void *fact_s = nullptr;       // general: S (c64); SPD: s = sqrt(lam) (float)
    double *fact_x = nullptr;     // FP64 copy of the returned X (for the adjoint residual)
    int fact_kind = 0;
    int fact_e = 0;
    double fact_norm = 0.0;
    // limit of the cooperative QR chase's inter-CTA waits (ns; 0 = 2 s)
    unsigned long long wait_ns = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // QR iteration: a second stream for the deferred window products, which
    // run while the next round of the chase does, and its ordering events
    // (chase done / deferred passes done, one pair per log buffer)
    cudaStream_t side = nullptr;
    cudaEvent_t qev[4] = {nullptr, nullptr, nullptr, nullptr};
    // captured launch sequences (CUDA graphs), keyed by what they depend on
    struct Graph {
        int tag;
        const void *key;
        int64_t n;
        int batch;
        uint64_t sig;  // anything else the captured launches depend on (0: nothing)
        cudaGraphExec_t exec;
        long long launches;
    };
    std::vector<Graph> graphs;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t body_stream = nullptr;  // captures the bodies of conditional nodes
    // tuning table (sqrtm_set_tuning), ascending n_max
    std::vector<sqrtm_tune_entry> tuning;
    // batched general path: device arena and pinned host buffer
    Buf bws;
    void *bpin = nullptr;
    size_t bpin_bytes = 0;
    // phases of the last batched-path graph (device clock): norms and casts,
    // Hessenberg reductions, QR rounds, Jacobi, triangular roots + X_0,
    // refinement loop; and the matrices it took (all, general)
    double bphase_ms[kBatchPhases] = {0, 0, 0, 0, 0};
    int bphase_count = 0, bphase_general = 0;
    // batched calls: worker handles, each on its own non-blocking stream
    char last_error[160] = {0};
    std::vector<sqrtm_handle_s *> workers;
    std::vector<cudaStream_t> worker_streams;
};

// Factors of one forward call, detached from the handle that computed them
// (sqrtm_factors_take): the device buffer that held them on the handle
// together with the pointers into it.
struct sqrtm_factors_s {
    Buf mem;
    int64_t n = -1;
    int kind = 0;
    int e = 0;
    double norm = 0.0;
    void *q = nullptr;     // general: Q (c64); SPD: V (float)
    void *s = nullptr;     // general: S (c64); SPD: s = sqrt(lam) (float)
    double *x = nullptr;   // FP64 X of that call
};

void drop_graphs(sqrtm_handle_t h, const void *lo, const void *hi);

inline int ensure(Buf &b, size_t bytes, sqrtm_handle_t owner = nullptr)
{
    if (b.bytes >= bytes) return 0;
    if (owner && b.p) drop_graphs(owner, b.p, (const char *)b.p + b.bytes);
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) return 7;
    b.bytes = bytes;
    return 0;
}

// bump allocator over a Buf, 256-byte aligned pieces
struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(void *p) : base((char *)p) {}
    template <class T> T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *r = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return r;
    }
    static size_t round(size_t bytes) { return (bytes + 255) & ~(size_t)255; }
};

// record the first failure of a call on the handle (for sqrtm_last_error)
void note_error(sqrtm_handle_t h, const char *what, int line, int code);

#define SQM_CU(call)                                          \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) {                              \
            note_error(h, cudaGetErrorName(_e), __LINE__, 7); \
            return 7;                                         \
        }                                                     \
    } while (0)


// The tuning entry for size n (nullptr without a table), and the automatic
// fields of opts resolved for size n: blks 0 -> tuned or 32, precision
// SQRTM_PREC_AUTO -> tuned or SQRTM_PREC_FP32.
const sqrtm_tune_entry *tune_for(sqrtm_handle_t h, int64_t n);
void apply_tuning(sqrtm_handle_t h, int64_t n, sqrtm_opts *o);

// The batched general path (batch.cu) for the matrices idx[0 .. count) of a
// batched call (n <= 46340 each); statuses into st_out[idx[i]].  Returns 0 or 7.
int batched_general(sqrtm_handle_t h, const int *idx, int count, const double *const *dA, const int64_t *n,
                    const int64_t *lda, double *const *dX, const int64_t *ldx, const sqrtm_opts &o, int *st_out);

// SPD path (Algorithm 3) and its FP64 counterpart, spd.cu
int spd_path(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, double tol, double *dX,
             int64_t ldx, const sqrtm_opts &o, sqrtm_info *info);
int spd_schur_fp64(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, double *dX,
                   int64_t ldx, const sqrtm_opts &o, sqrtm_info *info);
inline bool spd_enabled() { return true; }

// Enqueue `enqueue(stream)` on the handle's stream through a cached CUDA graph:
// the first call with a given (tag, key, n, batch) captures the launches on a
// private stream and instantiates them; later calls replay the executable
// graph.  The captured kernels must take all data-dependent arguments from
// device memory (descriptors), so a replay stays valid while `key` (the
// descriptor buffer) is the same allocation.  Returns 0 or 7.
int run_graph(sqrtm_handle_t h, int tag, const void *key, int64_t n, int batch,
              cudaError_t (*enqueue)(void *ctx, cudaStream_t s), void *ctx, uint64_t sig = 0);
// drop cached graphs whose key lies in [lo, hi) (a buffer being released)
void drop_graphs(sqrtm_handle_t h, const void *lo, const void *hi);
