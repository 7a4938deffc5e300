// launch.cuh -- kernel launch with programmatic dependent launch (PDL).
//
// Sweep kernels go out with programmatic stream serialization: each kernel
// may be scheduled before its predecessor on the stream has finished and
// waits for it inside the kernel (pdl_prologue in sweep_kernels.cuh, before
// its first read of mutable data).  That hides the launch and ramp-up of
// every kernel behind the one before it (~12 us per sweep at L = 4096 when
// it was introduced).  Stream capture records the dependencies as
// programmatic graph edges.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace xyk {

constexpr bool kUsePdl = true;

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), uint32_t grid, uint32_t block, size_t smem,
                       cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = kUsePdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace xyk
