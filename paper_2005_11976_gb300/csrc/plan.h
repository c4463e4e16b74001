// The plan object behind the opaque cyl_plan handle, and the host geometry helpers.
#pragma once

#include <mutex>
#include <vector>

#include "cylct_internal.h"

namespace cylct {

int set_error(int code, const char *msg);
int cuda_error(cudaError_t e, const char *what);

// geometry.cu
int validate_geom(const cyl_geom *geom);   // acquisition only (no grid, no pose)
void alignment_matrix(const cyl_pose &pose, double R[3][3]);   // X' = R (X - T)
int validate_scan(const cyl_grid *grid, const cyl_geom *geom, const cyl_pose *pose);
void build_grid(const cyl_grid &grid, const cyl_geom &geom, GridDev &g, std::vector<float2> &trig);
void build_views(const cyl_geom &geom, const cyl_pose &pose, std::vector<ProjGeom> &geo);
// Upper bound on the fraction of a scan's rays that meet the grid cylinder: per view the
// detector bounding box of the projected rim circles (the cylinder is their convex hull).
double hit_fraction_bound(const cyl_grid &grid, const cyl_geom &geom, const std::vector<ProjGeom> &geo);

// batch.cu: per round, the (scan, subset) items of a batched solve
void batch_rounds(const std::vector<int> &n_proj, int subset, int n_iter,
                  std::vector<BatchItem> &items, std::vector<int> &n_items, int &rounds);

// Buffers and settings of one SART solve.
struct SolveState {
    const void *sino = nullptr;
    cyl_dtype sino_t = CYL_F32;
    const void *x_proj = nullptr;  // volume the projector reads
    cyl_dtype x_proj_t = CYL_F32;
    float *x32 = nullptr;          // FP32 iterate (null in strict 16-bit mode)
    void *x16 = nullptr;           // 16-bit copy / iterate (null in FP32 mode)
    cyl_dtype x16_t = CYL_F16;
    int strict16 = 0;
    const void *w = nullptr;
    cyl_dtype w_t = CYL_F32;
    double lambda = 0.5;
    int clamp = 0;
    int subset = 1;
    int rec = 0;                   // subsets replay the pose's stored records (1) and gather per voxel (2)

    bool operator==(const SolveState &o) const
    {
        return sino == o.sino && sino_t == o.sino_t && x_proj == o.x_proj &&
               x_proj_t == o.x_proj_t && x32 == o.x32 && x16 == o.x16 && x16_t == o.x16_t &&
               strict16 == o.strict16 && w == o.w && w_t == o.w_t && lambda == o.lambda && clamp == o.clamp &&
               subset == o.subset && rec == o.rec;
    }
};

}  // namespace cylct

struct cyl_plan;

namespace cylct {

// Makes `dev` the current device for the guard's scope and restores the previous one.
// ok is false (err the CUDA error) when the switch failed; nothing may then be queued.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != dev && (err = cudaSetDevice(dev)) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
        }
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Plan kernels run on the plan's work stream, ordered after the caller's stream and
// before its later work: the plan's scratch and work counters serve one launch at a time.
struct OnPlanStream {
    cyl_plan *pl;
    cudaStream_t user;
    cudaError_t begin();
    cudaError_t end();
};

}  // namespace cylct

struct cyl_plan {
    int device = 0;
    cyl_grid grid{};
    cyl_geom geom{};
    cyl_pose pose{};
    std::vector<double> angles;
    std::vector<double> frames;    // n_proj x 12 of a general trajectory, or empty
    cylct::GridDev g{};
    int64_t n_vox = 0, n_pix = 0;
    size_t bytes = 0;

    cylct::ProjGeom *d_geo = nullptr;
    float2 *d_trig = nullptr;
    float4 *d_ray[3] = {nullptr, nullptr, nullptr};
    uint16_t *d_split = nullptr;   // [view][pixel][kSplit] cuts of each ray (per pose)
    int *d_sched = nullptr;        // work counters of the persistent kernels (kSched)
    // Compact plans (chosen at creation, where the grid surely leaves a quarter or more of
    // the detector dark) list each pose's rays of positive chord and keep records and cuts
    // for those rays only, at their list positions.
    bool use_list = false;
    uint32_t *d_act = nullptr;     // the list (plan ray indices), or null
    int64_t *d_act_off = nullptr;  // [n_proj + 1]: each view's start in the list
    int64_t *d_act_chunk = nullptr; // chunk counts / offsets of the list's construction
    int64_t n_listed = 0;          // rays listed for the current pose
    size_t ray_cap[3] = {0, 0, 0}, split_cap = 0, act_cap = 0;
    float *d_wscale = nullptr;
    float *d_q = nullptr;          // forward projections of one subset (FP32)
    size_t q_cap = 0;
    float2 *d_nd[2] = {nullptr, nullptr};   // (numerator, column sum) accumulators, per voxel
    int p_fp = 0, p_bp = 0;        // pieces per ray of the projector / back-projector (0: default)
    int p_sart = 0;                // pieces per ray of the fused SART kernel (0: default)
    bool fused = true;             // SART subsets in one launch (k_sart) instead of two
    // Stored segment records of the pose (records.cu; dense plans): rec_mode 0 (the
    // default) walks every ray in every subset; 1 writes each pose's pieces as records at
    // set-up, when they fit the device, and replays them in the one-launch subsets.
    int rec_mode = 0;
    int rec_lgP = cylct::kRecLgP;  // log2 of the runs per ray (replay lanes per ray)
    bool rec_ready = false;        // the records hold the current pose
    uint32_t *d_rcnt = nullptr;    // [view][pixel] pieces of each ray
    int32_t *d_ridx0 = nullptr;    // [view][pixel][runs] first voxel of each run
    int64_t *d_rrow = nullptr;     // first row of each task, and the total
    uint32_t *d_rec = nullptr;     // the records, rows of 32
    int *d_rbad = nullptr;         // set by the record walk if a count differs
    size_t rcnt_cap = 0, ridx0_cap = 0, rrow_cap = 0, rec_cap = 0, rbad_cap = 0;
    int64_t rec_rows = 0;
    // Eq. 7 with records: the numerator alone is reduced per subset (d_num, 4 ceil(V / 4)
    // floats); the column sums depend only on the pose and the subsets, so they are summed
    // once per pose and subset size (rinv_sub, 0: none; per view in FP32, d_den32, across
    // a subset's views in FP64, d_den64) and kept as reciprocals in d_rinv [subset][voxel].
    float *d_num = nullptr;
    float *d_rinv = nullptr;
    float *d_den32 = nullptr;
    double *d_den64 = nullptr;
    size_t num_cap = 0, rinv_cap = 0, den32_cap = 0, den64_cap = 0;
    int rinv_sub = 0;
    // The records' transpose (gather.cu; rec_mode 1, where it fits): per view and voxel the
    // pieces that cross the voxel, so that the subsets back-project by gathering per voxel
    // (vox_ready).  off [view][V + 1], ent (pixel, length) view after view, ebase per view.
    bool vox_ready = false;
    uint32_t *d_voff = nullptr, *d_vcnt = nullptr, *d_vcur = nullptr, *d_vtsum = nullptr;
    uint2 *d_vent = nullptr;
    int64_t *d_vebase = nullptr;
    size_t voff_cap = 0, vcnt_cap = 0, vcur_cap = 0, vtsum_cap = 0, vent_cap = 0, vebase_cap = 0;
    int64_t vox_entries = 0;
    float *d_x32 = nullptr;
    size_t x32_cap = 0;
    void *d_stage[4] = {nullptr, nullptr, nullptr, nullptr};  // sino, x0, w, x_out
    void *d_gamma = nullptr;       // scratch of cyl_estimate_gamma
    size_t gamma_cap = 0;
    size_t stage_cap[4] = {0, 0, 0, 0};

    cudaStream_t ws = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_geo = nullptr;
    void *h_geo = nullptr;         // pinned staging of the view tables (set_pose)

    bool timing = false;
    double kernel_ms[3] = {0, 0, 0};
    int64_t kernel_launches[3] = {0, 0, 0};
    std::vector<cudaEvent_t> events;
    size_t ev_used = 0;

    // captured sweeps, one per parity of the subset counter at the sweep's start
    cudaGraphExec_t gexec = nullptr, gexec_odd = nullptr;
    cylct::SolveState gkey{};
    // captured sweep with timing events (timing mode with graphs)
    cudaGraphExec_t gexec_timed = nullptr;
    cylct::SolveState gkey_timed{};
    size_t ev_timed = 0;           // events captured in gexec_timed (events[0 .. ev_timed))

    std::mutex mu;
    std::vector<void *> allocs;

    cylct::ScanDev scan_dev() const
    {
        cylct::ScanDev sd;
        sd.g = g;
        sd.trig = d_trig;
        sd.ray_a = d_ray[0];
        sd.ray_b = d_ray[1];
        sd.ray_c = d_ray[2];
        sd.split = d_split;
        sd.sched = d_sched;
        return sd;
    }
    cylct::RayList ray_list() const { return cylct::RayList{use_list ? d_act : nullptr, d_act_off}; }
    cylct::RecDev rec_dev() const { return cylct::rec_dev(scan_dev(), rec_lgP, d_rec, d_rrow, d_rcnt, d_ridx0); }
    cylct::VoxDev vox_dev() const
    {
        return cylct::VoxDev{d_vent, d_vebase, d_voff, n_vox, n_pix, g.eps};
    }

    template <class T> int alloc(T **p, size_t nbytes)
    {
        void *q = nullptr;
        if (cudaMalloc(&q, nbytes ? nbytes : 1) != cudaSuccess) {
            cudaGetLastError();
            return cylct::set_error(CYL_ENOMEM, "device allocation failed");
        }
        allocs.push_back(q);
        bytes += nbytes;
        *p = static_cast<T *>(q);
        return CYL_OK;
    }
    int init(const cyl_grid &gr, const cyl_geom &ge, const cyl_pose &po, int dev);
    // Upload view tables for `pose` and rebuild the ray records, on stream st.
    int upload_pose(const cyl_pose &po, cudaStream_t st);
    // Grow-only scratch buffer.
    int ensure(void **p, size_t &cap, size_t nbytes);
    void release(void **p, size_t &cap);
    // Records of the current pose (rec_mode 1): count (unless counted), size, write;
    // rec_ready tells whether they fit.  Synchronises st.
    int build_records(cudaStream_t st, bool counted = false);   // counted: d_rcnt holds the pose's counts
    int write_records(cudaStream_t st, bool counted);
    void free_records();
    // The records' transpose for the gather form (rec_mode 1); vox_ready tells whether it fits.
    int build_gather(cudaStream_t st);
    void free_gather();
    // Record buffers of a solve with subsets of `subset` views: 0 walk, 1 replay with the
    // pose's reciprocal column sums, 2 gather per voxel.
    int prepare_records(int subset, cudaStream_t st, int &rc);
    cudaEvent_t *next_events(int n);
    // Queue one sweep; `parity` is the subset counter's parity at its first subset.
    int queue_sweep(const cylct::SolveState &s, cudaStream_t st, bool timed, int parity);
    void drop_graphs();
    int tune(cudaStream_t st);
    int solve(const void *sino, cyl_dtype sino_t, const void *x0, const void *w,
              const cyl_sart_params &prm, void *x_out, cyl_dtype x_t, cudaStream_t user);
    ~cyl_plan();
};

inline cudaError_t cylct::OnPlanStream::begin()
{
    cudaError_t e = cudaEventRecord(pl->ev_in, user);
    return e == cudaSuccess ? cudaStreamWaitEvent(pl->ws, pl->ev_in, 0) : e;
}

inline cudaError_t cylct::OnPlanStream::end()
{
    cudaError_t e = cudaEventRecord(pl->ev_out, pl->ws);
    return e == cudaSuccess ? cudaStreamWaitEvent(user, pl->ev_out, 0) : e;
}
