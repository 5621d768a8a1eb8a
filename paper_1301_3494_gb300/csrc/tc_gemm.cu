// tcgen05 grouped GEMM (BF16 / TF32 operands, FP32 accumulation in TMEM).
#include "plans.h"

namespace pd {

bool tc_available() { return false; }

void run_gemm_tc(GemmBatch&, Num, const void*, long long, int, const void*, long long, int, void*, bool, unsigned*,
                 cudaStream_t) {
    throw Error{DMRG_ERR_STATE, "tensor-core GEMM engine not built"};
}

}  // namespace pd
