// Batched solve of many independent chains.
#include "solve.h"

extern "C" pmcmc_status pmcmc_solve_batched(pmcmc_ctx *c, int, const pmcmc_chain_desc *,
                                            const pmcmc_options *, pmcmc_result *, void *) {
    return pm::set_error(c, PMCMC_EUNSUPPORTED, "batched: not built yet");
}
