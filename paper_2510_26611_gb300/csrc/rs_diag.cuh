// Launch counting and opt-in event timing around kernel launches.
#pragma once

#include <cuda_runtime.h>

namespace rs {

// Adds n to the process-wide count of kernels launched by this library.
void note_launch(unsigned n = 1);

// Current timing mode (0 off, 1 major kernels, 2 all).
int timing_mode();

// Scope object around one kernel launch: counts it and, when timing is
// enabled, records a CUDA event pair on the launch stream.  `work` is the
// algorithmic flop (or byte) count of the launch, summed per kernel name.
// Timing mode 1 times only `major` launches (the pose kernels and the heavy
// build kernels); mode 2 times every launch.  With allow_events false the launch
// is only counted (no CUDA events are created).
class KernelTimer {
  public:
    KernelTimer(const char* name, cudaStream_t st, double work = 0.0, bool major = true,
                bool allow_events = true);
    ~KernelTimer();
    KernelTimer(const KernelTimer&) = delete;
    bool active() const { return active_; }
    void set_work(double w) { work_ = w; }
    KernelTimer& operator=(const KernelTimer&) = delete;

  private:
    const char* name_;
    cudaStream_t st_;
    double work_;
    cudaEvent_t a_{}, b_{};
    bool active_ = false;
};

}  // namespace rs
