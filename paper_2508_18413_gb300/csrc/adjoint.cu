// Adjoint of a chain functional at the converged fixed point (reverse dense scan).
#include "solve.h"

extern "C" pmcmc_status pmcmc_adjoint(pmcmc_ctx *c, const pmcmc_target *, const pmcmc_options *,
                                      int, const void *, const void *, const unsigned char *,
                                      const void *, const double *, const void *, size_t,
                                      double *, void *) {
    return pm::set_error(c, PMCMC_EUNSUPPORTED, "adjoint: not built yet");
}
