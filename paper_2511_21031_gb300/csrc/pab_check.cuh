// Checked build: bounds checks on the kernels' global-memory accesses.
//
// Built with -DPAB_CHECKED (the library libpab_checked.so), every global-memory
// access of the kernels goes through PAB_LD / PAB_ST / PAB_AT with the length
// of its buffer: an index outside [0, length) is not accessed (a load gives
// zero), and the first such index of a translation unit is recorded with its
// source line and bound in a device word of that unit, which
// pab_check_report (pab_measure.h) reads and clears.  It stands in for a
// memory checker on machines where none can run; it changes no result of a
// correct kernel.  Without PAB_CHECKED the macros are the plain accesses.
//
// Each .cu file with kernels includes this header once and places
// PAB_CHECK_UNIT(name) at file scope, which defines the host-side reader
// pab::check_fetch_name of its record (a zero record in an unchecked build).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "pab_internal.h"

#ifdef PAB_CHECKED
namespace {
__device__ pab::CheckRecord g_pab_check;

// The zero of a buffer's element type (what a skipped load gives).
template <class T>
__device__ __forceinline__ typename std::remove_cv<T>::type pab_zero(const T *)
{
    return typename std::remove_cv<T>::type();
}

__device__ __forceinline__ bool pab_check_index(long long i, long long n, int line)
{
    if (i >= 0 && i < n)
        return true;
    if (atomicAdd(&g_pab_check.count, 1u) == 0u) {
        g_pab_check.line = line;
        g_pab_check.index = i;
        g_pab_check.bound = n;
    }
    return false;
}
}  // namespace

// value of p[i] (zero of its type when i is outside [0, n))
#define PAB_LD(p, i, n) \
    (pab_check_index((long long)(i), (long long)(n), __LINE__) ? (p)[i] : pab_zero(p))
// p[i] = v (skipped when i is outside [0, n))
#define PAB_ST(p, i, n, v)                                                  \
    do {                                                                    \
        if (pab_check_index((long long)(i), (long long)(n), __LINE__))      \
            (p)[i] = (v);                                                   \
    } while (0)
// __ldcg(p + i) (read through L2), zero outside [0, n)
#define PAB_LDCG(p, i, n) \
    (pab_check_index((long long)(i), (long long)(n), __LINE__) ? __ldcg((p) + (i)) : pab_zero(p))
// __ldg(p + i) (read-only path), zero outside [0, n)
#define PAB_LDG(p, i, n) \
    (pab_check_index((long long)(i), (long long)(n), __LINE__) ? __ldg((p) + (i)) : pab_zero(p))
// &p[i] for an atomic (i clamped to 0 when outside [0, n): the caller's update then lands on a
// valid element, and the record says where the index went wrong)
#define PAB_AT(p, i, n) (&(p)[pab_check_index((long long)(i), (long long)(n), __LINE__) ? (i) : 0])

#define PAB_CHECK_UNIT(name)                                                             \
    namespace pab {                                                                      \
    void check_fetch_##name(CheckRecord *r, bool clear)                                  \
    {                                                                                    \
        cudaMemcpyFromSymbol(r, g_pab_check, sizeof(CheckRecord));                       \
        if (clear) {                                                                     \
            const CheckRecord z = {0u, 0, 0, 0};                                         \
            cudaMemcpyToSymbol(g_pab_check, &z, sizeof(CheckRecord));                    \
        }                                                                                \
    }                                                                                    \
    }
#else
#define PAB_LD(p, i, n) ((p)[i])
#define PAB_ST(p, i, n, v) ((p)[i] = (v))
#define PAB_LDCG(p, i, n) __ldcg((p) + (i))
#define PAB_LDG(p, i, n) __ldg((p) + (i))
#define PAB_AT(p, i, n) (&(p)[i])
#define PAB_CHECK_UNIT(name)                                  \
    namespace pab {                                           \
    void check_fetch_##name(CheckRecord *r, bool)             \
    {                                                         \
        r->count = 0u;                                        \
        r->line = 0;                                          \
        r->index = 0;                                         \
        r->bound = 0;                                         \
    }                                                         \
    }
#endif
