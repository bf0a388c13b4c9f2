// Launch interface of the pose kernels, shared with the batching runtime.
#pragma once

#include "rs_common.cuh"

namespace rs {

struct EvalLaunch {
    ProteinView prot;
    LigandView lig;
    const double* rot = nullptr;    // quaternions [P][4] or rotation vectors [P][3]
    const double* trans = nullptr;  // [P][3]
    long long P = 0;
    double* E = nullptr;
    uint8_t* flags = nullptr;
    double* gt = nullptr;           // gradient outputs (gradient launches)
    double* gw = nullptr;
    int PB = 0;                     // poses per block (0: heuristic)
    int grid = 0;                   // CTAs (0: persistent, fill the GPU)
    bool events = true;             // allow timing events (off for the no-allocation path)
    const uint8_t* skip = nullptr;  // [P] nonzero: skip the pose, leave its outputs untouched
};

rs_status launch_prep_ligand(int L, const double* xyz, const double* q, float4* y, double* y64,
                             double* q64, cudaStream_t st, bool events = true);
rs_status launch_eval(const EvalLaunch& a, bool grad, cudaStream_t st);
size_t ligand_scratch_bytes(int L);
LigandView carve_ligand(void* base, int L);

}  // namespace rs
