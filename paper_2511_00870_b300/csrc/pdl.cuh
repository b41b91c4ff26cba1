// Device side of programmatic dependent launch (see launch_pdl): wait for the
// predecessor grid's completion and memory, and allow the dependent grid to
// launch. Both are no-ops for a kernel launched without the attribute.
#pragma once

namespace pnp {
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
}  // namespace pnp
