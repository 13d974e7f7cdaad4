// Owner records of the sort-free back end: one 32-bit word per (phase,
// array, index) cell.  Shared by the interpreter and, as text, by the
// per-protocol kernels compiled at run time.
//
// Definition 1 asks, per cell, whether some access writes it and whether two
// different threads access it.  A record keeps exactly that:
//   bits 0..29  the first accessor's tid + 1 (0 while none), set once by CAS
//   bit 30      a second, different thread has accessed the cell
//   bit 31      some access wrote the cell
// so the cell is racy iff bits 30 and 31 are both set.  Records only gain
// bits during a launch; an access whose bits a (possibly stale) copy of the
// record already implies changes nothing and is skipped.  A read-only cell
// saturates with its second distinct reader, a written one with the write and
// the second thread, so hot cells stop costing atomics almost at once.
// Thread ids stay below 2^27 (a preparation limit), so tid + 1 fits.
#pragma once

namespace drf {

constexpr uint32_t kOwnerRep = 0x3FFFFFFFu;
constexpr uint32_t kOwnerMulti = 1u << 30;
constexpr uint32_t kOwnerWritten = 1u << 31;

__device__ __forceinline__ bool owner_racy(uint32_t r) { return (r & kOwnerMulti) && (r & kOwnerWritten); }

// One access by thread `tid` (w: it writes).  `cur` is a copy of the record
// read through L1 (it may be stale; the record itself only gains bits).
__device__ __forceinline__ void owner_put(uint32_t *cell, uint32_t cur, uint32_t tid, uint32_t w)
{
    const uint32_t me = tid + 1;
    if (cur == 0) {
        const uint32_t old = atomicCAS(cell, 0u, me | (w << 31));
        if (old == 0) return;
        cur = old;
    }
    uint32_t need = 0;
    if (!(cur & kOwnerMulti) && (cur & kOwnerRep) != me) need |= kOwnerMulti;
    if (w && !(cur & kOwnerWritten)) need |= kOwnerWritten;
    if (need) atomicOr(cell, need);
}

// Accesses of two or more different threads to one cell at once (a warp
// whose lanes agree on the cell): the cell is multi-owner.
__device__ __forceinline__ void owner_put_many(uint32_t *cell, uint32_t cur, uint32_t any_write)
{
    const uint32_t need = kOwnerMulti | (any_write ? kOwnerWritten : 0u);
    if ((cur & need) != need) atomicOr(cell, need);
}

}  // namespace drf
