// Backward render (replaced below by the real kernels).
#include "ss3d_internal.cuh"

void ss_launch_raster_bwd(const ss_ws_view&, const ss_layout&, const ss_bwd_args&, cudaStream_t) {}
void ss_launch_project_bwd(const ss_ws_view&, const ss_layout&, const ss_bwd_args&, cudaStream_t) {}
