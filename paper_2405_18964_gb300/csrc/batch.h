// batch.h -- shared frequency solves of the serving loop (internal; api.cu).
#pragma once
#include <stddef.h>

#include "pint.h"

struct pint_batcher_s;

struct pint_batch_stats {
  long long batches;       // shared frequency solves run
  long long member_solves; // member applies they served (sum of batch sizes)
  long long frequencies;   // frequencies solved in them
  int max_members;         // largest batch
};

pint_batcher_s* batcher_create();
void batcher_destroy(pint_batcher_s* b);
// A handle whose frequency solves run in the shared context of its group.
pint_status member_create(pint_batcher_s* b, const pint_params* p, void* stream, pint_handle* out);
void member_destroy(pint_handle h);
// Bracket a member's solve (its group's batches wait, bounded, for members in a solve).
void member_solve_begin(pint_handle h);
void member_solve_end(pint_handle h);
void batcher_get_stats(pint_batcher_s* b, pint_batch_stats* out);
void shared_estimates(const pint_params* p, size_t* member_bytes, size_t* per_freq_bytes);
