// Host-side state of a multi-event batch (shared by batch.cu and persistent.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/glasma.h"
#include "internal.h"

struct BatchEvent {
    glasma_params gp;
    cpic_params pp;
    int id;
    int n;
    size_t ns;
    int n_steps, n_form, np, acc_rows;
    double a_fm, a_gev, dtau, mass;
    void* buf[3];        // rotating: iteration k reads buf[k % 3], writes buf[(k + 1) % 3]
    void* init_buf;
    void* rec;           // gather records of the record push, REC_STRIDE groups per cell
    int* occ;            // occupancy stamps of the record push, one per cell
    void* frc;           // contracted fields of the split push, 6 particle planes
    void* part_base;
    void* part_init;
    size_t part_bytes;
    glasma::PartHost P;
    double* acc;
    double* mon;
    long long ic_fails;
    double ic_mean;
    int ic_max;
};

struct glasma_batch {
    int prec = 0, E = 0, nmax = 0, max_iter = 0;
    cudaStream_t st = nullptr;
    size_t fft_work = 0;
    std::vector<BatchEvent> ev;   // ordered by step count, descending
    std::vector<int> pos;         // caller's event index -> position in ev
    void* step_args = nullptr;    // [max_iter][E] StepArgs
    void* push_args = nullptr;    // [max_iter][E] PushArgs
    void* tiles_dev = nullptr;    // TileItem list, grouped by event (persistent path)
    void* gtiles_dev = nullptr;   // TileItem list of the chosen field variant (graph and eager paths)
    int fvar = 0;                 // FP32 field tile variant of the graph and eager paths
    int pvar = 0;                 // batched push kernel of the graph and eager paths
    bool any_sub = false;         // some event takes several particle steps per field step or the CIC gather
    // pushes on a second stream (graph and eager modes): push k after field k, field k+2
    // after push k (the buffer field k+2 writes is the one push k reads as fo)
    bool two_streams = false;
    cudaStream_t st2 = nullptr;
    std::vector<cudaEvent_t> sev;  // [2 * max_iter + 1]: after field k, after push k, after the restore
    // graph timing: event-record nodes around every field launch of the batched path
    bool timing = false;
    std::vector<cudaEvent_t> tev;  // [2 * max_iter]: start, end of field launch k
    int tev_used = 0;              // pairs recorded by the last enqueue
    void* pitems_dev = nullptr;   // PushItem list, grouped by event
    void* scratch = nullptr;      // initial-condition / sort scratch
    std::vector<int> tiles_upto, gtiles_upto, pitems_upto, active;
    bool initialised = false, graph_ready = false;
    cudaGraphExec_t exec = nullptr;
    // persistent mode
    void* pers_ctrl = nullptr;    // barrier counters + error word + per-iteration prefixes (device)
    int pers_blocks = 0;
    unsigned long long pers_spin = 1ull << 24;  // grid-barrier polls (~100 ns each) before giving up
    bool pers_launched = false;   // the error word is meaningful only after a persistent run
};

void glasma_set_error(const char* msg);
glasma_status batch_run_persistent(glasma_batch* b);
bool batch_timed_out(glasma_batch* b);  // reads (and clears) the persistent kernel's error word
void batch_free_persistent(glasma_batch* b);
