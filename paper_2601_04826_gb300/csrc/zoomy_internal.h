// zoomy_internal.h -- the context object behind the opaque zoomy_ctx handle (internal).
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/zoomy.h"

#define ZOOMY_MAX_LEVEL 4
#define ZOOMY_MESH_ENSEMBLE 3  // internal kind of an ensemble context (zoomy_ensemble_create)

namespace zoomy {
struct DevCtl;
constexpr int NPARTIAL = 1024;  // blocks of the fixed-order FP64 mass sum
}  // namespace zoomy

struct zoomy_ctx {
    // mesh
    int kind = 0, dim = 1;
    int64_t nx = 0, ny = 1, nc = 0;
    double dx = 1, dy = 1, area_const = 1, min_delta = 1;
    int bc[4] = {0, 0, 0, 0};
    std::vector<double> bed_host;   // caller's cell order
    std::vector<int64_t> perm;      // triangles: perm[new] = caller index
    // device / stream
    cudaStream_t stream = nullptr;
    int device = 0, nsm = 1;
    // model
    bool model_ok = false;
    int level = 0, dtype = 0, nv = 0;
    zoomy_friction fric = {0, 0.0, 0.0, 1.0, 0.0};
    double g = 9.81, cfl = 0.45, hdry = 0.0;
    int src_implicit = 0;  // 0: explicit Newtonian + implicit bottom stress; 1: friction fully implicit
    int order = 1;         // space order: 1, or 2 (MUSCL, fv_order2.cu; 1D and structured 2D)
    int vam = 0;           // 1: the non-hydrostatic VAM predictor-corrector (vam.cu), 1D FP64
    double *vam_sys = nullptr, *vam_p = nullptr;  // its pressure system (block rows, reduction arrays), p
    // device buffers owned by the context
    void *bed_dev = nullptr;
    void *q1 = nullptr;
    size_t q1_bytes = 0;
    void *qdev_host = nullptr;      // device copy used by zoomy_step_host
    size_t qdev_host_bytes = 0;
    zoomy::DevCtl *ctl = nullptr;      // step control: wave-speed slots, time, sticky status
    zoomy::DevCtl *ctl_aux = nullptr;  // scratch of the synchronous reductions
    double *partials = nullptr;
    // structured 2D decomposition (rows per warp segment, warps per block)
    int rows_per_warp = 0, warps_per_block = 4;  // rows_per_warp 0: rows_per_warp_for()
    int launch_1d = 0, warps_per_cta_1d = 0;     // zoomy_tune_1d
    // stage-kernel profiling (zoomy_profile_enable)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_events;  // pool, reused
    std::vector<int> prof_kind;            // stage of each recorded (start, stop) pair
    size_t prof_used = 0;                  // events in use
    // learned closure (fv_closure.cu): level-1 model closed with predicted level-4 moments
    void *closure_d = nullptr;
    void *closure_pred = nullptr;  // predicted closed moments of the current stage input [6][nx ny]
    void *closure_tc = nullptr;    // the network in the tcgen05 operand layout
    int closure_engine = 0;        // 0: tcgen05 (tensor memory), 1: mma.sync
    int closure_schedule = 0;      // 0: network on every stage input, 1: once per step on Q^n
    bool closure_on = false;
    double closure_lambda = 0.0;
    // ensemble (fv_ensemble.cu)
    void *ens = nullptr;
    // triangle mesh (device)
    int32_t *tri_nbr_d = nullptr;   // [3][nc] neighbour cell or -1
    float *tri_geo_d = nullptr;     // per cell-face normals and lengths / area
    double *tri_area_d = nullptr;   // [nc]
};

namespace zoomy {
// Segment height of the structured 2D row-marching kernels when none was set: about
// warps_per_sm warps per SM over the grid (30-column strips), within [8, 64] rows.
inline int rows_per_warp_for(int64_t nx, int64_t ny, int nsm, int warps_per_sm)
{
    const int64_t want = (int64_t)(nsm > 0 ? nsm : 1) * warps_per_sm;
    const int64_t H = ((nx + 29) / 30) * ny / want;
    return (int)(H < 8 ? 8 : (H > 64 ? 64 : H));
}

zoomy_status set_error(zoomy_status st, const char *fmt, ...);
zoomy_status cuda_fail(cudaError_t e, const char *where);
zoomy_status ctx_init_device(zoomy_ctx *c);
zoomy_status read_status(zoomy_ctx *c, double *t_total);
// record a profiling event before / after a stage launch (no-op when profiling is off)
zoomy_status prof_mark(zoomy_ctx *c, int stage, bool start);
zoomy_status check_step_args(zoomy_ctx *c, const void *Q, int64_t ld, double dt, int32_t nsteps, const char *who);
// friction parameters accepted by zoomy_model_set and zoomy_step_noalloc: a known kind, rho > 0 and
// C, nu, manning_n >= 0 (negative values would run as anti-damping)
inline bool friction_ok(const zoomy_friction &f)
{
    return f.kind >= 0 && f.kind <= 2 && f.rho > 0.0 && f.C >= 0.0 && f.nu >= 0.0 && f.manning_n >= 0.0;
}
// triangle meshes (fv_tri.cu)
zoomy_status create_tri_mesh(const zoomy_mesh_desc *d, void *stream, zoomy_ctx **out);
void tri_free(zoomy_ctx *c);
void ens_free(zoomy_ctx *c);
// learned closure (fv_closure.cu)
zoomy_status closure_run_steps(zoomy_ctx *c, float *Q, int64_t ld, double dt, int nsteps);
zoomy_status closure_max_wavespeed(zoomy_ctx *c, const float *Q, int64_t ld, double *out);
// VAM predictor-corrector (vam.cu)
zoomy_status vam_run_steps(zoomy_ctx *c, double *Q, int64_t ld, double dt, int nsteps);
zoomy_status closure_upload(zoomy_ctx *c, const float *params, const float *in_scale, const float *out_scale);
zoomy_status tri_run_steps(zoomy_ctx *c, float *Q, int64_t ld, double dt, int nsteps);
}  // namespace zoomy
