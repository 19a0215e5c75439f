// Batched apply over work queues: the interface between the batch handle (batch.cu) and the
// persistent-queue launch sequence (batch_queue.cu).
#pragma once
#include <string>
#include <vector>

#include "ifgf_internal.cuh"

namespace ifgf {

// Settings of the queue sequence (ifgf_batch_set).
struct QueueConfig {
    int cones_per_item = 16;      // parent cones per propagation work item (multiple of 4)
    int blocks_per_sm = 0;        // resident blocks of the persistent propagation kernel (0: occupancy limit)
    int64_t wait_limit = 1 << 24; // polls of a dependency counter before IFGF_ERR_TIMEOUT
    int withhold = -1;            // test only: problem * 64 + level whose first item is never counted
};

struct BatchQueue;

// Whether the plans can run as one queue sequence: mixed precision, orders (3,5,5), one density
// each, one device. Otherwise *why says what is missing.
bool queue_eligible(const std::vector<Plan*>& plans, const int32_t* nrhs, std::string* why);
// Work lists and coefficient storage of the batch (device memory of its own; plan-time work).
BatchQueue* queue_create(const std::vector<Plan*>& plans);
void queue_destroy(BatchQueue* q);
// Points the sequence at the callers' densities and outputs (a small copy on stream s when they
// changed since the last call).
void queue_set_io(BatchQueue* q, const void* const* dens, void* const* outs, cudaStream_t s);
// Builds the propagation queue for the settings (host work and device allocation: call it
// outside a stream capture).
void queue_prepare(BatchQueue* q, const QueueConfig& c);
// Enqueues the whole sequence on s (stream capture or direct): counter reset, permutation in,
// near field, LevelDEvaluations, the propagation, interpolation, permutation out.  With branch
// streams (fork/join events ev: one fork, then one per branch) the propagation is each plan's own
// per-level kernels, plan i on branch i mod branches.size(), instead of the persistent queue.
void queue_record(BatchQueue* q, const QueueConfig& c, cudaStream_t s, const std::vector<cudaStream_t>* branches = nullptr,
                  const std::vector<cudaEvent_t>* ev = nullptr);
// Queue items of the propagation (for tests and the withhold index) and the first item of a
// (problem, level) pair, -1 if that level has no propagation.
int64_t queue_items(const BatchQueue* q);
int64_t queue_first_item(const BatchQueue* q, int problem, int level);
// Sticky status of the last sequences (IFGF_OK or IFGF_ERR_TIMEOUT); synchronises the device.
int queue_status(BatchQueue* q);

}  // namespace ifgf
