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
    void* ws = nullptr;             // scratch of the cell-grouped Tucker path (NULL: one pass
    size_t ws_bytes = 0;            //   per block of poses, no scratch)
};

rs_status launch_prep_ligand(int L, const double* xyz, const double* q, float4* y, float2* yd, double* y64,
                             double* q64, cudaStream_t st, bool events = true);
rs_status launch_eval(const EvalLaunch& a, bool grad, cudaStream_t st);
// The long-range and short-range passes of launch_eval without the local-box flag
// pass: the cell-grouped path for large Tucker calls, else the per-block kernels.
rs_status launch_eval_paths(const EvalLaunch& a, bool grad, cudaStream_t st);
// Local-box handles: OR the out-of-grid flag into flags[p] for every pose (not skipped)
// with an atom whose interpolation cell lies outside the handle's box (no-op for
// other handles or NULL flags).
rs_status launch_box_flags(const ProteinView& P, const LigandView& lig, const double* rot, const double* trans,
                           long long Ptot, bool rotvec, const uint8_t* skip, uint8_t* flags, cudaStream_t st);
size_t ligand_scratch_bytes(int L);
// Cell-grouped Tucker path (rs_sorted.cu): scratch for P poses (capped at one chunk)
// and the number of poses one chunk of ws_bytes holds.
size_t sorted_scratch_bytes(long long P, int L, int n, bool grad);
long long sorted_chunk_poses(size_t ws_bytes, int L, int n, bool grad);
rs_status launch_sorted(const EvalLaunch& a, bool grad, cudaStream_t st);
// Finite-difference forces (Eq. differ_ligand) and their rigid-cluster resultants
// (Eq. Field_Xcenter, Eq. Field_phi) of a.P poses given by rotation vectors (a.rot)
// on the cell-grouped path; a.ws/a.ws_bytes as for launch_sorted (sized by
// sorted_fd_scratch_bytes), vbuf: fd_pose_bytes(sorted_fd_chunk_poses(...)) bytes.
struct FdOut {
    double* E;
    uint8_t* flags;  // may be NULL
    double* F;       // [P][3] sum_l F_l
    double* F0;      // [P][3] radial resultant
    double* Fphi;    // [P][3] tangential resultant at radius r0
    double* M;       // [P][3] sum_l r_l x F_l
};
long long sorted_fd_chunk_poses(size_t ws_bytes, int L, int n);
size_t sorted_fd_scratch_bytes(long long P, int L, int n);
size_t fd_pose_bytes(long long PC);
rs_status launch_sorted_fd(const EvalLaunch& a, double h, double r0, void* vbuf, const FdOut& o, cudaStream_t st);
LigandView carve_ligand(void* base, int L);

}  // namespace rs
