// Tensor-core contraction (a) with fused quadrature (b): placeholder until the
// tcgen05 kernel lands.
#include "blast_internal.h"

int launch_contract_tc(blast_plan *, ReqDev *, int, const int *, int, void *, void *, cudaStream_t)
{
    return BLAST_ENOBASIS;
}
