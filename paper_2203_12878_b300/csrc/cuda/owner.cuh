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

// The bits an access by thread `tid` (w: it writes) adds to a non-empty
// record `cur`: multi-owner when the record's first accessor is another
// thread, written when it writes.  Zero when `cur` already implies the access.
__device__ __forceinline__ uint32_t owner_need(uint32_t cur, uint32_t tid, uint32_t w)
{
    uint32_t need = 0;
    if (!(cur & kOwnerMulti) && (cur & kOwnerRep) != tid + 1) need |= kOwnerMulti;
    if (w && !(cur & kOwnerWritten)) need |= kOwnerWritten;
    return need;
}

// The record after one access by the thread whose tid + 1 is `t1`
// (`wbit`: kOwnerWritten when it writes, else 0), for a record no other
// thread updates meanwhile (a plain read and write): an empty record takes
// the thread as first accessor, a non-empty one gains the bits the access
// implies.  Branch-free; the result equals `cur` when nothing changes.
__device__ __forceinline__ uint32_t owner_merge(uint32_t cur, uint32_t t1, uint32_t wbit)
{
    const uint32_t multi = (cur & kOwnerRep) != t1 ? kOwnerMulti : 0u;
    return cur == 0u ? (t1 | wbit) : (cur | wbit | multi);
}

// One access by thread `tid` (w: it writes).  `cur` is a copy of the record
// read earlier in this launch (it may be out of date; the record itself only
// gains bits, so an old copy costs at most a redundant update).  An
// empty copy claims the record (first accessor) by compare-and-swap.
// Returns true when this call turned the record from zero into non-zero.
__device__ __forceinline__ bool owner_put(uint32_t *cell, uint32_t cur, uint32_t tid, uint32_t w)
{
    if (cur == 0) {
        const uint32_t old = atomicCAS(cell, 0u, (tid + 1) | (w << 31));
        if (old == 0) return true;
        cur = old;
    }
    const uint32_t need = owner_need(cur, tid, w);
    if (need) atomicOr(cell, need);
    return false;
}

// Accesses of two or more different threads to one cell at once (a warp
// whose lanes agree on the cell): the cell is multi-owner.  Returns true when
// the copy was zero (this call may have turned the record non-zero).
__device__ __forceinline__ bool owner_put_many(uint32_t *cell, uint32_t cur, uint32_t any_write)
{
    const uint32_t need = kOwnerMulti | (any_write ? kOwnerWritten : 0u);
    if ((cur & need) != need) atomicOr(cell, need);
    return cur == 0;
}

// Marks the block of record `off` in the touch bitmap (one bit per
// 2^block_log records).  A record turns non-zero exactly once per launch,
// through an update whose copy was zero, and only that update marks its
// block: every block holding a non-zero record is marked, and the scan that
// clears the table reads exactly the marked blocks.  A plain reduction:
// reading the word first would put a dependent load on the claiming path.
__device__ __forceinline__ void owner_touch(uint32_t *touch, unsigned long long off, int block_log)
{
    const unsigned long long bid = off >> block_log;
    atomicOr(touch + (bid >> 5), 1u << (uint32_t)(bid & 31));
}

}  // namespace drf
