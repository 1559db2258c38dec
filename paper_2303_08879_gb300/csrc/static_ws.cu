// static_ws.cu -- fock_diag_probs_static: the all-detected forward walk with
// its scratch in a fixed device array owned by the library, for callers that
// cannot allocate device memory themselves.
//
// The array below is device memory reserved when the library is loaded onto a
// GPU and kept until the process exits.  Host code must not use its name as a
// pointer: on the host that name only stands in for the device symbol.  Every
// call looks the device address up with cudaGetSymbolAddress on the current
// GPU (a lookup, no allocation), so an address never outlives the context it
// came from (after cudaDeviceReset the module is loaded again, possibly at
// another address); the walk kernel then receives that address exactly as it
// would receive a caller-supplied workspace.
#include <cuda_runtime.h>

#include "fk_internal.h"
#include "../../include/fockdiag.h"

namespace {

constexpr size_t kStaticBytes = (size_t)FK_STATIC_WORKSPACE_BYTES;

static __device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

// Device address of g_static_ws in the current GPU's context.
int static_workspace(void **out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_ws) != cudaSuccess || !p) return FK_ECUDA;
    *out = p;
    return FK_OK;
}

}  // namespace

extern "C" int fock_diag_probs_static(int batch, const fk_c128 *A, const fk_c128 *b,
                                      const fk_c128 *c, int M, const int *cutoffs,
                                      fk_c128 *probs, unsigned flags, void *stream,
                                      int *host_status)
{
    using namespace fk;
    if (batch < 1 || !A || !b || !c || !probs) return FK_EINVAL;
    DiagShape sh;
    int rc = build_diag_shape(M, cutoffs, !(flags & FK_FLAG_B_ZERO), &sh);
    if (rc) return rc;
    DiagLayout lay;
    rc = diag_layout(sh, batch, false, flags, &lay);
    if (rc) return rc;
    if (lay.total > kStaticBytes) return FK_EWORKSPACE;
    void *ws = nullptr;
    rc = static_workspace(&ws);
    if (rc) return rc;
    // The launcher clears the control block (barrier counters, status word)
    // with cudaMemsetAsync before the kernel; the rest of the array needs no
    // initial value (every amplitude is written before it is read).
    rc = launch_diag_forward(sh, batch, flags, A, b, c, probs, ws, lay, stream);
    if (rc || !host_status) return rc;
    return read_status(ws, stream, host_status);
}
