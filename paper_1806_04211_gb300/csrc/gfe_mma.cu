// tcgen05 tensor-core block multiply-add (placeholder until the kernel lands).
#include "gfe_internal.h"

namespace gfe {

bool mad_tc(const Launch &, int64_t, int64_t, int64_t, const void *, int64_t, const void *, int64_t,
            const void *, int64_t, void *, int64_t) {
    return false;
}

}  // namespace gfe
