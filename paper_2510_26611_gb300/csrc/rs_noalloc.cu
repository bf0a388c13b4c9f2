// Pose energies without any device allocation at call time.
//
// rs_energy_poses keeps its per-call scratch (the ligand re-centred on its
// geometric centre, in FP32 and FP64) in a context buffer that grows with
// cudaMalloc.  Some callers cannot allow that: a service thread that must never
// trigger cudaMalloc/cudaFree (they can synchronise the whole device and stall
// other users' streams), or a plug-in inside a host application that owns all
// device memory through its own pool and forbids libraries from allocating on
// their own.  This file gives them a variant whose scratch is a fixed array in
// the library's own device image, sized for the largest ligand it accepts.
#include <mutex>

#include "rs_common.cuh"
#include "rs_eval.cuh"

namespace rs {
namespace {

constexpr int kNoAllocMaxL = 4096;
constexpr int kMaxDevices = 64;
// Prepared-ligand layout (see carve_ligand): float4 y[L], float2 yd[L][3] (coordinate
// pairs), double y64[L][3], double q64[L], each part 256-byte aligned.
constexpr size_t kNoAllocBytes = ((size_t)kNoAllocMaxL * 16 + 255) / 256 * 256 +
                                 2 * (((size_t)kNoAllocMaxL * 24 + 255) / 256 * 256) +
                                 ((size_t)kNoAllocMaxL * 8 + 255) / 256 * 256;

// One copy per GPU that loads the library; it lives until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).
// Looked up once per device; in host code the array's name is only a host-side
// stand-in, so the address must come from cudaGetSymbolAddress.
rs_status scratch_for(int device, void** out) {
    if (device < 0 || device >= kMaxDevices) {
        set_error("rs_energy_poses_noalloc: device %d out of range", device);
        return RS_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("rs_energy_poses_noalloc: cudaGetSymbolAddress failed: %s",
                      cudaGetErrorString(e));
            cudaGetLastError();
            return RS_ERR_CUDA;
        }
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return RS_OK;
}

// The caller's buffers must be memory this GPU can address: device memory on
// `device`, or managed memory.  A host pointer (or another GPU's memory) handed to
// the kernels would fault and poison the context, so it is refused here, on the
// host, before anything is launched.  cudaPointerGetAttributes allocates nothing.
rs_status check_on_device(const void* p, int device, const char* what) {
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("rs_energy_poses_noalloc: %s is not a CUDA pointer (%s)", what,
                  cudaGetErrorString(e));
        return RS_ERR_INVALID;
    }
    if (a.type == cudaMemoryTypeManaged) return RS_OK;
    if (a.type != cudaMemoryTypeDevice || a.device != device) {
        set_error("rs_energy_poses_noalloc: %s must be device memory on GPU %d "
                  "(pointer type %d on device %d)", what, device, (int)a.type, a.device);
        return RS_ERR_INVALID;
    }
    return RS_OK;
}

}  // namespace
}  // namespace rs

extern "C" rs_status rs_energy_poses_noalloc(const rs_protein* prot, int32_t L,
                                             const double* lig_xyz, const double* lig_q,
                                             int64_t P, const double* quat, const double* trans,
                                             double* E_out, uint8_t* flags_out, void* stream) {
    using namespace rs;
    clear_error();
    RS_CHECK_ARG(prot, "rs_energy_poses_noalloc: NULL protein");
    if (prot->view.box) {
        set_error("rs_energy_poses_noalloc: local-box handles are not supported (use rs_energy_poses)");
        return RS_ERR_UNSUPPORTED;
    }
    RS_CHECK_ARG(L >= 1, "rs_energy_poses_noalloc: L=%d must be >= 1", L);
    if (L > kNoAllocMaxL) {
        set_error("rs_energy_poses_noalloc: L=%d exceeds the fixed scratch limit of %d atoms",
                  L, kNoAllocMaxL);
        return RS_ERR_UNSUPPORTED;
    }
    RS_CHECK_ARG(P >= 0 && P <= 0x7fffffffLL, "rs_energy_poses_noalloc: P=%lld out of range",
                 (long long)P);
    if (P == 0) return RS_OK;
    RS_CHECK_ARG(lig_xyz && lig_q && quat && trans && E_out,
                 "rs_energy_poses_noalloc: NULL input or output pointer");
    RS_TRY_CUDA(cudaSetDevice(prot->device));
    RS_TRY(check_on_device(lig_xyz, prot->device, "lig_xyz"));
    RS_TRY(check_on_device(lig_q, prot->device, "lig_q"));
    RS_TRY(check_on_device(quat, prot->device, "quat"));
    RS_TRY(check_on_device(trans, prot->device, "trans"));
    RS_TRY(check_on_device(E_out, prot->device, "E_out"));
    if (flags_out) RS_TRY(check_on_device(flags_out, prot->device, "flags_out"));
    void* scratch = nullptr;
    RS_TRY(scratch_for(prot->device, &scratch));
    cudaStream_t st = (cudaStream_t)stream;
    LigandView lig = carve_ligand(scratch, L);
    RS_TRY(launch_prep_ligand(L, lig_xyz, lig_q, (float4*)lig.y, (float2*)lig.yd, (double*)lig.y64,
                              (double*)lig.q64, st, false));
    EvalLaunch a;
    a.prot = prot->view;
    a.lig = lig;
    a.rot = quat;
    a.trans = trans;
    a.P = P;
    a.E = E_out;
    a.flags = flags_out;
    a.events = false;
    return launch_eval(a, false, st);
}
