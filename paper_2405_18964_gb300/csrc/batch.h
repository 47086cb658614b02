// batch.h -- shared frequency solves (internal; api.cu implements, serve.cpp uses).
#pragma once
#include <stddef.h>

#include "pint.h"

pint_batcher_s* batcher_create();
void batcher_destroy(pint_batcher_s* b);
// A handle whose frequency solves run in the shared context of its subgroup.
pint_status member_create(pint_batcher_s* b, const pint_params* p, void* stream, pint_handle* out);
void member_destroy(pint_handle h);
void batcher_get_stats(pint_batcher_s* b, pint_group_stats* out);
void shared_estimates(const pint_params* p, size_t* member_bytes, size_t* per_freq_bytes);
