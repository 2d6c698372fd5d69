// Kernel launches with programmatic dependent launch (PDL).
//
// A V-cycle is thousands of short dependent kernels (every tree depth of every slab
// solve is one), so the gap between one kernel's end and the next one's start is a
// large part of its time.  launch_k() queues a kernel with programmatic stream
// serialisation: the next kernel may be scheduled while this one drains, and its
// blocks wait in griddepcontrol.wait until the previous grid has completed and its
// memory is visible.  Every kernel therefore calls pdl_entry(), which waits first and
// then lets its own dependent be scheduled, before it reads or writes anything another
// kernel writes (most begin with it), so the ordering is the same as a plain stream's
// (and transitively so: a grid completes only after its own wait).
#pragma once

#include <cuda_runtime.h>

#include <utility>

#include "device.h"

namespace stmg {

__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch_cfg(bool overlap, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = overlap ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // status: the caller's cudaGetLastError(); the caller also counts the launch
  cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
  launch_cfg(launch_overlap(), kern, grid, block, smem, st, std::forward<Args>(args)...);
}

// Always with programmatic stream serialisation: for a kernel that reads nothing a kernel
// writes before it calls pdl_entry() (its prologue may then overlap the previous kernel).
template <typename... KArgs, typename... Args>
inline void launch_k_overlap(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             Args&&... args) {
  launch_cfg(true, kern, grid, block, smem, st, std::forward<Args>(args)...);
}

}  // namespace stmg
