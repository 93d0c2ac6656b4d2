// Tensor-core (sm_103a tcgen05) path of the jump term and of the Sylvester updates.
#include "lb_internal.cuh"

size_t mixed_bytes(int, int) { return 0; }
int mixed_prepare(lb_handle_s* h, cudaStream_t) { h->mixed_ready = false; return 0; }
int jump_mixed(lb_handle_s*, cudaStream_t, const cplx*, cplx*, double) { return -1; }
int trisylv_mixed(lb_handle_s*, cudaStream_t, cplx*, double) { return -1; }
void mixed_release(lb_handle_s*) {}
lb_handle_s::~lb_handle_s() { mixed_release(this); }
