// tet.cu -- unstructured tetrahedral meshes (placeholder until the tet path lands).
#include "internal.cuh"

namespace cgk {

cg_status tet_build(cg_mesh *, int64_t, const double *, int64_t, const int32_t *) {
    return fail(CG_EINVAL, "tetrahedral meshes are not built yet");
}
void tet_release(cg_mesh *) {}
cg_status tet_locate_launch(cg_mesh *, int64_t, const double *, int, const double *, int32_t *,
                            uint32_t *, unsigned long long *, cudaStream_t) {
    return fail(CG_EINVAL, "tetrahedral meshes are not built yet");
}
cg_status diffuse_tet_run(cg_mesh *, int, double *, const cg_params *, cg_report *, cudaStream_t) {
    return fail(CG_EINVAL, "tetrahedral meshes are not built yet");
}

}  // namespace cgk
