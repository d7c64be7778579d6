// Internal interface of the batch engine (solver.cu) for the serving loop (server.cu): solves
// whose set-up ran on their own plan stream join one engine thread that iterates every joined
// solve together (two preconditioner passes and one tile kernel per iteration, replayed from a
// captured graph) and hands each back when its stopping rule holds.
#pragma once
#include <cstddef>
#include <cstdint>

#include "rlobpcg.h"

namespace rl {

struct BatchEngine;
struct BatchSolve;

int batch_engine_create(int device, BatchEngine** out);
void batch_engine_stats(BatchEngine* e, rlobpcg_engine_stats* out);
// every submitted solve must have been waited for
void batch_engine_destroy(BatchEngine* e);
// real FP64, block <= 5, n <= 512, at most 200 iterations, no locking, SVQB or residual refresh
bool batch_request_eligible(int64_t n, int k, int dtype, const rlobpcg_opts& o);
// device bytes a batched solve adds to its plan while it iterates
size_t batch_extra_bytes(int64_t m, int64_t n, int b);
// sketch, factor, start block and first Rayleigh-Ritz step on the plan's stream; A (device) must
// stay valid until batch_solve_finish
int batch_solve_setup(rlobpcg_plan_t p, const double* A, int64_t lda, BatchSolve** out);
void batch_solve_submit(BatchEngine* e, BatchSolve* s);
// blocks until the engine has retired the solve; its status
int batch_solve_wait(BatchSolve* s);
// outputs on the plan's stream (as rlobpcg_solve); releases the handle
int batch_solve_finish(BatchSolve* s, double* sigma, void* V, void* U, double* resid, rlobpcg_info* info);

}  // namespace rl
