// batch.cuh -- device descriptor of one job of the batched engine and the
// launcher of its persistent kernel (kernels_batch.cu).
#pragma once
#include "common.cuh"

namespace hdmd {

enum JobKind { JOB_MD = 0, JOB_FIRE = 1 };
enum JobStatus { JOB_ACTIVE = 0, JOB_DONE = 1, JOB_NOT_CONVERGED = 2, JOB_ERROR = 3 };

// One job: its arrays (Dev, with one gather buffer: gs[1] == gs[0],
// gd[1] == gd[0]), its progress and, for FIRE, the FIRE scalar state.  The
// kernel resumes a job where the previous launch left it.
struct BatchJob {
    Dev dv;
    int kind;          // JobKind
    int status;        // JobStatus
    int mixed;         // FP32 pair arithmetic (until the FIRE polish switch)
    int phase64;       // pair arithmetic currently FP64
    int built;         // lists exist for the current positions
    int force_valid;   // dv.F holds the forces at the current positions
    int lgG;           // lanes per atom (log2), set per dimension by the host
    int error;         // ErrBits seen
    long long steps_done, nsteps;   // MD progress
    double dt;                      // MD time step
    double fire[FS_COUNT];          // FIRE state and parameters
    double sums[kNRed];             // last reduction (Red slots)
    long long builds;
};

struct BatchCtl {
    int first;            // this dimension's slice of the order array: [first, first + njobs)
    int njobs;
    int next;             // work-queue ticket
    long long budget;     // iterations (FIRE) or steps (MD) per job per launch; 0 = to the end
};

constexpr int kBatchNT = 256;       // threads per job block
constexpr int kBatchWideNT = 512;   // threads per block of the large jobs
constexpr int kBatchWideN = 4096;   // jobs with more atoms run in the wide blocks

// persistent kernel over the jobs of dimension D listed in order[0..ctl->njobs),
// and the timing probe of the lanes-per-atom autotuner (builds the job's lists
// if needed, then evaluates its forces reps times with the job's lgG)
#define HDMD_BATCH_DECLARE(D)                                                          \
    void launch_batch_d##D(BatchJob *jobs, const int *order, BatchCtl *ctl, int grid,  \
                           cudaStream_t s);                                            \
    void launch_batch_wide_d##D(BatchJob *jobs, const int *order, BatchCtl *ctl,       \
                                int grid, cudaStream_t s);                             \
    void launch_batch_probe_d##D(BatchJob *job, int reps, cudaStream_t s);
HDMD_BATCH_DECLARE(2)
HDMD_BATCH_DECLARE(3)
HDMD_BATCH_DECLARE(4)
HDMD_BATCH_DECLARE(5)
HDMD_BATCH_DECLARE(6)
HDMD_BATCH_DECLARE(7)
HDMD_BATCH_DECLARE(8)
HDMD_BATCH_DECLARE(9)
HDMD_BATCH_DECLARE(10)
#undef HDMD_BATCH_DECLARE

}  // namespace hdmd
