// Device side of the batched pose launch, shared by rs_batch.cu (captured batches)
// and rs_serve.cu (the serving loop): pair descriptors, work items and the
// persistent kernel that takes items from a device counter.
#pragma once

#include <algorithm>
#include <vector>

#include "rs_common.cuh"
#include "rs_pose_dev.cuh"

namespace rs {
namespace {

struct BatchItem {
    int pair;
    int PB;
    long long p0;
};

template <int RP, int NT>
__global__ void __launch_bounds__(NT) k_eval_batch(const PairDesc* __restrict__ pairs,
                                                   const BatchItem* __restrict__ items, int nitems,
                                                   int* __restrict__ counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int cur;
    __shared__ __align__(16) PairDesc pd;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
        __syncthreads();
        const int it = cur;
        if (it >= nitems) break;
        const BatchItem bi = items[it];
        const int* src = (const int*)(pairs + bi.pair);
        for (int e = threadIdx.x; e < (int)(sizeof(PairDesc) / sizeof(int)); e += NT)
            ((int*)&pd)[e] = src[e];
        __syncthreads();
        wform_block<RP, false, NT>(pd.prot, pd.lig, pd.rot, pd.trans, pd.P, bi.PB, bi.p0, pd.E,
                                   pd.flags, nullptr, nullptr, smem);
    }
}

struct Shape {
    int nt;      // threads per CTA
    int atoms;   // target atoms per item
};

int pb_for(int L, int atoms) { return std::min(128, std::max(1, atoms / L)); }

template <int RP, int NT>
size_t batch_smem(const std::vector<int>& Ls, int atoms) {
    size_t m = 0;
    for (int L : Ls) m = std::max(m, wform_smem<RP, false, NT>(pb_for(L, atoms), L));
    return m;
}

}  // namespace

// Block shape picked for a padded rank by the batch autotuner (default if untuned).
void batch_shape_for(int RP, int* nt, int* atoms);

}  // namespace rs
