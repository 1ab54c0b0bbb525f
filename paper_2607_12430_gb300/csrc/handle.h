// handle.h -- the library handle (workspace, saved factors, events) and
// small host helpers shared by the C-ABI translation units.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "internal.h"
#include "../../include/sqrtm_mp.h"
#include "../../include/sqrtm_mp_steps.h"

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
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
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

inline int ensure(Buf &b, size_t bytes)
{
    if (b.bytes >= bytes) return 0;
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

#define SQM_CU(call)                              \
    do {                                          \
        cudaError_t _e = (call);                  \
        if (_e != cudaSuccess) return 7;          \
    } while (0)


// SPD path (Algorithm 3) and its FP64 counterpart, spd.cu
int spd_path(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, double tol, double *dX,
             int64_t ldx, const sqrtm_opts &o, sqrtm_info *info);
int spd_schur_fp64(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, double *dX,
                   int64_t ldx, const sqrtm_opts &o, sqrtm_info *info);
inline bool spd_enabled() { return true; }
