// Level-scheduled triangular-solve state shared by the solve and refinement.
#pragma once
#include "common.cuh"

namespace kc {

struct Solver {
    const kc_pattern* P = nullptr;
    int2* tasks = nullptr;
    int64_t ntasks = 0;
    int rpt = 64;
    int maxr = 0;
    int* ready = nullptr;
    unsigned* cnt = nullptr;
    unsigned* gcnt = nullptr;
    double* acc = nullptr;
    unsigned long long* ticket = nullptr;
    int* status = nullptr;
    double* y = nullptr;
    float2* xf = nullptr;  // FP32 form: x as (hi, lo) pairs
    int nrhs_cap = 0;
    long long spin = 4000000000LL;
};

kc_status build_tasks(const kc_pattern* P, int rpt, Arena& A, cudaStream_t s, int2** tasks_out, int64_t* ntasks_out,
                      int* max_row_out, bool adaptive = false);
kc_status solver_init(Solver& S, const kc_pattern* P, int nrhs_cap, const kc_opts* o, Arena& A, cudaStream_t s);
template <typename T>
kc_status solver_apply(Solver& S, const T* val, const double* diag, double diag_fallback, const double* rhs,
                       double* z, int nrhs, cudaStream_t s);
kc_status solver_check(Solver& S, cudaStream_t s);
// point-major copies with stride >= nrhs (0: nrhs); to_point_major zero-fills the padding
kc_status to_point_major(const double* b, const int32_t* perm, int64_t N, int nrhs, double* out, cudaStream_t s,
                         int stride = 0);
kc_status from_point_major(const double* xp, const int32_t* perm, int64_t N, int nrhs, double* x, cudaStream_t s,
                           int stride = 0);

}  // namespace kc
