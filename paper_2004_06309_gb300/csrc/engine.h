// Internal interface between a solver context (capi.cu) and the serving layer
// (server.cpp): analysis kept apart from device residency, and the slot engine of
// the continuous pseudo-block FGMRES.  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <string>

#include "../../include/hz.h"
#include "host.h"

namespace hz_engine {

enum { SLOT_FREE = 0, SLOT_RUN = 1, SLOT_DONE = 2 };

// Host analysis of a mesh (assembly pattern, decomposition, coarse space, symbolic
// factorisations): frequency independent, reusable for any number of contexts.
hz_status analyse_problem(const hz_mesh_desc* md, const hz_options* op, hz::HostProblem& P, std::string& err);

// Device bytes a context of P holds after hz_factor (persistent) and the transient
// frontal workspace of the factorisation on top of it.
void plan_bytes(const hz::HostProblem& P, const hz_options& op, int64_t& persistent, int64_t& transient);

// Context on the calling thread's current device from an analysed problem (P is not
// modified).  op->hbm_budget caps every allocation of the context, factor included.
hz_status create(const hz::HostProblem& P, int order, const hz_options* op, hz_ctx** out, std::string& err);

int64_t device_bytes(const hz_ctx* c);

// Slot engine (requires options.block_size > 1).
int slot_count(const hz_ctx* c);
int slot_state(const hz_ctx* c, int i);
bool slots_running(const hz_ctx* c);
hz_status slot_point_source(hz_ctx* c, int i, const double xyz[3]);
hz_status slot_start(hz_ctx* c, int i, double tol, int64_t tag);
void slots_issue(hz_ctx* c);
hz_status slots_complete(hz_ctx* c);
hz_status slot_harvest(hz_ctx* c, int i, void* x, bool on_device, hz_rhs_info* info);
void slot_reset(hz_ctx* c, int i);        // frees a slot whatever its state

}  // namespace hz_engine

namespace hz {
long long launch_count();   // process-wide count of the library's kernel launches
}
