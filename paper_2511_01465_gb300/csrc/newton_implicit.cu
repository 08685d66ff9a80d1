// newton_implicit.cu -- instantiations of the persistent small-state Newton
// kernel for the implicit step maps of Sec. 3.4 (backward Euler and the
// trapezoidal rule) and for the stiff test systems of Sec. 4.2 (Dahlquist,
// Robertson).
//
// The implicit maps run in the fused kernel (newton_fused.cuh; the explicit
// Euler ones in the three-phase kernel): either only needs a map
// whose eval(x_{n-1}, x_n) yields the scan element of step n; for backward
// Euler that element is (M_n^{-1}, -M_n^{-1} h_n) with M_n = I - h Jf(x_n)
// (eqs. 3.16-3.19), built by BackwardEulerMap in systems.cuh; TrapezoidMap
// builds the trapezoidal rule's.  Both rules also run with the FP32
// delta-form and the float-float scans (the fused reduced-precision kernel,
// newton_fused_mixed.cuh);
// the batched and adjoint entry points are explicit-only.
#include "newton_small.cuh"

namespace pitn_host {

int select_implicit_kernel(int system_id, int method, int precision, pitn::SmallKernel* K) {
    using namespace pitn;
    if (precision == PITN_PREC_MIXED_FP32 && method == PITN_STEP_TRAPEZOID) {
        switch (system_id) {
        case PITN_DAHLQUIST: *K = small_kernel_of<TrapezoidMap<DahlquistRhs>, kVarFusedMixed>(); return PITN_OK;
        case PITN_ROBERTSON: *K = small_kernel_of<TrapezoidMap<RobertsonRhs>, kVarFusedMixed>(); return PITN_OK;
        case PITN_VDP: *K = small_kernel_of<TrapezoidMap<VdpRhs>, kVarFusedMixed>(); return PITN_OK;
        case PITN_LOGISTIC: *K = small_kernel_of<TrapezoidMap<LogisticRhs>, kVarFusedMixed>(); return PITN_OK;
        default: return PITN_EUNSUPPORTED;
        }
    }
    if (precision == PITN_PREC_FP64_FF && method == PITN_STEP_TRAPEZOID) {
        switch (system_id) {
        case PITN_DAHLQUIST: *K = small_kernel_of<TrapezoidMap<DahlquistRhs>, kVarFusedFF>(); return PITN_OK;
        case PITN_ROBERTSON: *K = small_kernel_of<TrapezoidMap<RobertsonRhs>, kVarFusedFF>(); return PITN_OK;
        case PITN_VDP: *K = small_kernel_of<TrapezoidMap<VdpRhs>, kVarFusedFF>(); return PITN_OK;
        case PITN_LOGISTIC: *K = small_kernel_of<TrapezoidMap<LogisticRhs>, kVarFusedFF>(); return PITN_OK;
        default: return PITN_EUNSUPPORTED;
        }
    }
    if (precision == PITN_PREC_MIXED_FP32) {
        // backward Euler with the FP32 delta-form scan: the residual and the
        // inverse of I - h Jf stay FP64, the folds, scans and replay FP32
        if (method != PITN_STEP_BACKWARD_EULER) return PITN_EUNSUPPORTED;
        switch (system_id) {
        case PITN_DAHLQUIST: *K = small_kernel_of<BackwardEulerMap<DahlquistRhs>, kVarFusedMixed>(); return PITN_OK;
        case PITN_ROBERTSON: *K = small_kernel_of<BackwardEulerMap<RobertsonRhs>, kVarFusedMixed>(); return PITN_OK;
        case PITN_VDP: *K = small_kernel_of<BackwardEulerMap<VdpRhs>, kVarFusedMixed>(); return PITN_OK;
        case PITN_LOGISTIC: *K = small_kernel_of<BackwardEulerMap<LogisticRhs>, kVarFusedMixed>(); return PITN_OK;
        default: return PITN_EUNSUPPORTED;
        }
    }
    if (precision == PITN_PREC_FP64_FF) {
        // backward Euler with the float-float scan: the residual, the inverse
        // and the update in FP64, the dense folds, scans and replay in pairs
        // of floats
        if (method != PITN_STEP_BACKWARD_EULER) return PITN_EUNSUPPORTED;
        switch (system_id) {
        case PITN_DAHLQUIST: *K = small_kernel_of<BackwardEulerMap<DahlquistRhs>, kVarFusedFF>(); return PITN_OK;
        case PITN_ROBERTSON: *K = small_kernel_of<BackwardEulerMap<RobertsonRhs>, kVarFusedFF>(); return PITN_OK;
        case PITN_VDP: *K = small_kernel_of<BackwardEulerMap<VdpRhs>, kVarFusedFF>(); return PITN_OK;
        case PITN_LOGISTIC: *K = small_kernel_of<BackwardEulerMap<LogisticRhs>, kVarFusedFF>(); return PITN_OK;
        default: return PITN_EUNSUPPORTED;
        }
    }
    if (precision != PITN_PREC_FP64) return PITN_EUNSUPPORTED;
    if (method == PITN_STEP_BACKWARD_EULER) {
        switch (system_id) {
        case PITN_DAHLQUIST: *K = small_kernel_of<BackwardEulerMap<DahlquistRhs>, kVarFused>(); return PITN_OK;
        case PITN_ROBERTSON: *K = small_kernel_of<BackwardEulerMap<RobertsonRhs>, kVarFused>(); return PITN_OK;
        case PITN_VDP: *K = small_kernel_of<BackwardEulerMap<VdpRhs>, kVarFused>(); return PITN_OK;
        case PITN_LOGISTIC: *K = small_kernel_of<BackwardEulerMap<LogisticRhs>, kVarFused>(); return PITN_OK;
        default: return PITN_EUNSUPPORTED;
        }
    }
    if (method == PITN_STEP_TRAPEZOID) {
        switch (system_id) {
        case PITN_DAHLQUIST: *K = small_kernel_of<TrapezoidMap<DahlquistRhs>, kVarFused>(); return PITN_OK;
        case PITN_ROBERTSON: *K = small_kernel_of<TrapezoidMap<RobertsonRhs>, kVarFused>(); return PITN_OK;
        case PITN_VDP: *K = small_kernel_of<TrapezoidMap<VdpRhs>, kVarFused>(); return PITN_OK;
        case PITN_LOGISTIC: *K = small_kernel_of<TrapezoidMap<LogisticRhs>, kVarFused>(); return PITN_OK;
        default: return PITN_EUNSUPPORTED;
        }
    }
    if (method == PITN_STEP_EULER) {
        switch (system_id) {
        case PITN_DAHLQUIST: *K = small_kernel_of<EulerMap<DahlquistRhs>, kVarPlain>(); return PITN_OK;
        case PITN_ROBERTSON: *K = small_kernel_of<EulerMap<RobertsonRhs>, kVarPlain>(); return PITN_OK;
        default: return PITN_EUNSUPPORTED;
        }
    }
    return PITN_EUNSUPPORTED;
}

}  // namespace pitn_host
