"""Model of the BDL-tree's forest bookkeeping — TEST INFRASTRUCTURE.

The BDL-tree (paper, Section 5) keeps static kd-trees in slots i = 0, 1, ...
with capacity 2^i * X, plus a buffer tree of capacity X.  This model tracks
*which point ids* live in which slot and in the buffer; it builds no trees,
because the exact k-NN answer of the forest equals the k-NN of its live point
set (Section 5 "Data-Parallel k-NN"), which `oracle.knn` computes directly.

Insert_L (Section 5 "Parallel Batch Insertion"; Appendix A.2, Algorithm 3):
  * F is the bitmask of occupied slots.
  * |P| mod X points of the batch go to the buffer.  If the buffer then holds
    X or more points, X of them are taken out and join P.
  * F_new = F + floor(|P| / X) (+1 when the buffer overflowed).
  * Slots set in F but not in F_new are destroyed; slots set in F_new but not
    in F are built from the destroyed trees' points plus batch points.
Erase_L (Appendix A.3, Algorithm 4):
  * erase the points from every tree (and the buffer);
  * gather the points of every tree left with fewer than half of its capacity;
  * reinsert them with Insert_L.

Readings where the paper is silent (this model takes each of them as stated):
  * which batch points go to the buffer: the last |P| mod X of the batch, in
    batch order (a new batch is in input order; a reinserted set is in
    ascending id order);
  * which buffer points overflow: the X smallest ids of the buffer after the
    remainder was added; they follow the batch points in the pool;
  * how points are distributed over several new trees: new slots are filled in
    increasing slot order; slot j first takes every not-yet-taken destroyed
    tree of a lower slot, then pool points in order up to its capacity 2^j X;
    the highest new slot takes all pool points that remain (after deletions it
    can hold fewer than its capacity, never fewer than half);
  * erase matches points by bitwise-equal float32 coordinates and removes all
    live copies; absent points are ignored;
  * "fewer than half of its capacity" is 2 * live < 2^i X; the buffer tree is
    exempt.
"""
from __future__ import annotations

import numpy as np


class BDLModel:
    def __init__(self, dim: int, X: int):
        assert X >= 1
        self.dim = dim
        self.X = X
        self.F = 0                      # bitmask of occupied slots
        self.slots: dict[int, list[int]] = {}
        self.buffer: list[int] = []     # sorted ids
        self.coords: dict[int, bytes] = {}
        self.points: list[np.ndarray] = []   # id -> float32 row
        self.next_id = 0

    # ------------------------------------------------------------------ helpers
    def capacity(self, i: int) -> int:
        return (1 << i) * self.X

    def live_ids(self) -> list[int]:
        out = list(self.buffer)
        for ids in self.slots.values():
            out += ids
        return sorted(out)

    def size(self) -> int:
        return len(self.buffer) + sum(len(v) for v in self.slots.values())

    def slot_sizes(self) -> dict[int, int]:
        return {i: len(v) for i, v in sorted(self.slots.items())}

    def slot_of(self) -> np.ndarray:
        """slot index per id; -2 for the buffer, -1 for erased ids."""
        s = np.full(self.next_id, -1, np.int64)
        for i, ids in self.slots.items():
            s[ids] = i
        s[self.buffer] = -2
        return s

    # ------------------------------------------------------------------ Insert_L
    def insert(self, pts) -> np.ndarray:
        pts = np.ascontiguousarray(pts, dtype=np.float32).reshape(-1, self.dim)
        ids = list(range(self.next_id, self.next_id + len(pts)))
        for i, row in zip(ids, pts):
            self.points.append(row.copy())
            self.coords[i] = row.tobytes()
        self.next_id += len(pts)
        self._insert_ids(ids)
        return np.asarray(ids, np.int64)

    def _insert_ids(self, P: list[int]) -> None:
        X = self.X
        s = len(P)
        q, r = divmod(s, X)
        batch, to_buffer = P[: s - r], P[s - r:]
        merged = sorted(self.buffer + to_buffer)
        if len(merged) >= X:
            overflow, self.buffer = merged[:X], merged[X:]
            q += 1
        else:
            overflow, self.buffer = [], merged
        pool = batch + overflow
        assert len(pool) == q * X
        F_new = self.F + q
        consumed = [i for i in range(F_new.bit_length() + 1) if (self.F >> i) & 1 and not (F_new >> i) & 1]
        created = [j for j in range(F_new.bit_length() + 1) if (F_new >> j) & 1 and not (self.F >> j) & 1]
        taken: set[int] = set()
        pos = 0
        new_slots: dict[int, list[int]] = {}
        for n, j in enumerate(created):
            members: list[int] = []
            for i in consumed:
                if i < j and i not in taken:
                    members += self.slots[i]
                    taken.add(i)
            if n == len(created) - 1:
                members += pool[pos:]
                pos = len(pool)
            else:
                need = self.capacity(j) - len(members)
                assert need > 0
                members += pool[pos:pos + need]
                pos += need
            new_slots[j] = members
        assert taken == set(consumed), "every destroyed tree feeds a new one"
        assert pos == len(pool)
        for i in consumed:
            del self.slots[i]
        self.slots.update(new_slots)
        self.F = F_new

    # ------------------------------------------------------------------ Erase_L
    def erase(self, pts) -> int:
        pts = np.ascontiguousarray(pts, dtype=np.float32).reshape(-1, self.dim)
        keys = {row.tobytes() for row in pts}
        removed = 0

        def keep(i):
            return self.coords[i] not in keys

        for slot in list(self.slots):
            before = len(self.slots[slot])
            self.slots[slot] = [i for i in self.slots[slot] if keep(i)]
            removed += before - len(self.slots[slot])
        before = len(self.buffer)
        self.buffer = [i for i in self.buffer if keep(i)]
        removed += before - len(self.buffer)
        R: list[int] = []
        for slot in sorted(self.slots):
            if 2 * len(self.slots[slot]) < self.capacity(slot):
                R += self.slots.pop(slot)
                self.F &= ~(1 << slot)
        self._insert_ids(sorted(R))
        return removed

    # ------------------------------------------------------------------ queries
    def live_arrays(self):
        """(points (L, dim) float32, ids (L,) int64) of the live set, by id."""
        ids = self.live_ids()
        if not ids:
            return np.zeros((0, self.dim), np.float32), np.zeros(0, np.int64)
        return np.stack([self.points[i] for i in ids]), np.asarray(ids, np.int64)

    def check_invariants(self) -> None:
        """Every live id in exactly one place; occupied slots >= half capacity."""
        seen: set[int] = set()
        for i, ids in self.slots.items():
            assert (self.F >> i) & 1
            assert 0 < len(ids) <= self.capacity(i)
            assert 2 * len(ids) >= self.capacity(i)
            assert not seen.intersection(ids)
            seen.update(ids)
        assert not seen.intersection(self.buffer)
        assert len(self.buffer) < self.X
        assert bin(self.F).count("1") == len(self.slots)
