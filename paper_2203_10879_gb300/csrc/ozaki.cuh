// FP64 products emulated on the bf16 tensor cores (Ozaki-style splitting).
#pragma once
#include "common.cuh"

namespace sr {

constexpr int kOzakiMaxSlices = 12;
constexpr bool kOzakiBuilt = false;

struct OzakiWork {
    int nmax = 0;
};

inline cudaError_t ozaki_alloc(OzakiWork &w, int nmax, int) { w.nmax = nmax; return cudaSuccess; }
inline void ozaki_free(OzakiWork &) {}

template <class EP>
sr_status ozaki_gemm(schur_refine_ctx *, cudaStream_t, OzakiWork &, bool, int, int, int, const double *, int, const double *, int,
                     EP, double *, int *, int)
{
    return SR_ERR_UNSUPPORTED;
}

}  // namespace sr
