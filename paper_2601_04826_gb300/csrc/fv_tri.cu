// fv_tri.cu -- triangle meshes (cell-centric gather kernel over Morton-ordered cells).
#include "zoomy_internal.h"

namespace zoomy {

zoomy_status create_tri_mesh(const zoomy_mesh_desc *, void *, zoomy_ctx **)
{
    return set_error(ZOOMY_EINVAL, "zoomy_mesh_create: triangle meshes are not available in this build");
}

void tri_free(zoomy_ctx *c)
{
    cudaFree(c->tri_nbr_d);
    cudaFree(c->tri_geo_d);
    cudaFree(c->tri_area_d);
}

zoomy_status tri_run_steps(zoomy_ctx *, float *, int64_t, double, int)
{
    return set_error(ZOOMY_EINVAL, "triangle meshes are not available in this build");
}

}  // namespace zoomy
