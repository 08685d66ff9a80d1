// fkpp.cu -- Newton solve for the Fisher-KPP method-of-lines systems (d >= 3).
#include "common.cuh"
#include "solver.h"

namespace pitn_host {

int fkpp_solve(const SolveIO&, double, int64_t, int, double, int, const pitn_options&, cudaStream_t,
               SolveOutcome*) {
    return PITN_EUNSUPPORTED;
}

}  // namespace pitn_host

extern "C" {

int pitn_solve_batch(int, int64_t, const double*, const double*, const double*, const int64_t*, int,
                     double, int, double*, int64_t*, int32_t*, int32_t*, double*,
                     const pitn_options*) {
    return PITN_EUNSUPPORTED;
}

int pitn_backward(int, int64_t, const double*, const double*, const double*, const int64_t*, int,
                  const double*, const double*, const double*, int, double*, double*,
                  const pitn_options*) {
    return PITN_EUNSUPPORTED;
}

}
