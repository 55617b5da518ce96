"""The mbarrier protocol of the pipelined scan kernels, replayed on the CPU.

`scan_tiles` (long texts) and `scan_units` (batches) hand tiles from a
producer warp to the filtering warps through three mbarriers per buffer:
`full` (the copy landed), `ready` (realigned and packed) and `empty` (every
filtering warp is done). Tile k uses buffer k % nb and waits on phase k / nb
of each barrier, by parity, exactly as the kernels do; the producer polls
its two duties (hand over the next landed tile; refill the buffer of tile
issued - nb once it is released), and a batch ends with a closing
descriptor and meets its filtering warps at machine changes. A model of an
mbarrier (count, pending arrivals, phase) runs both sides with random copy
latencies and warp speeds and checks: nothing deadlocks, no buffer is
refilled while a warp still reads it, every warp reads the tile it expects,
and every copy has landed when the work ends."""
import random


class Bar:
    def __init__(self, count):
        self.count = count
        self.pending = count
        self.phase = 0

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count

    def test(self, parity):
        """mbarrier.test_wait.parity: the phase with this parity completed."""
        return (self.phase & 1) != parity


def simulate(tiles, machs=None, nb=3, ncw=16, seed=0):
    """One CTA: `tiles` tiles (batch form when `machs` gives each tile's
    machine: a closing descriptor ends the work, warps meet at changes)."""
    rng = random.Random(seed)
    batch = machs is not None
    full = [Bar(1) for _ in range(nb)]
    ready = [Bar(1) for _ in range(nb)]
    empty = [Bar(ncw) for _ in range(nb)]
    meet = Bar(ncw)
    in_buf = [None] * nb
    released = {}
    inflight = []
    t = 0
    total = None

    def claim(k):   # returns whether tile k exists
        b = k % nb
        if in_buf[b] is not None and in_buf[b] != "end":
            assert released.get(in_buf[b], 0) == ncw, "buffer refilled while in use"
        if k >= tiles:
            in_buf[b] = "end"
            return False
        in_buf[b] = k
        inflight.append((k, t + rng.randint(1, 6)))
        return True

    issued = prepped = 0
    while issued < min(nb, tiles + (1 if batch else 0)) and total is None:
        if not claim(issued):
            total = issued
        issued += 1
    if not batch:
        total = tiles
    producer_done = False
    warps = [{"k": 0, "busy": 0, "mach": None, "meet": 0, "state": "wait", "done": False}
             for _ in range(ncw)]
    for step in range(1, 500_000):
        t += 1
        for x in list(inflight):
            if x[1] <= t:
                inflight.remove(x)
                full[x[0] % nb].arrive()
        if not producer_done:
            b = prepped % nb
            if prepped < issued:
                if prepped == total:                   # closing descriptor: no copy
                    ready[b].arrive()
                    producer_done = True
                elif full[b].test((prepped // nb) & 1):
                    assert in_buf[b] == prepped
                    ready[b].arrive()
                    prepped += 1
            elif prepped == total:
                producer_done = True
            if (not producer_done and issued >= nb and issued < tiles + (1 if batch else 0)
                    and (total is None or issued < total)
                    and empty[issued % nb].test((issued // nb - 1) & 1)):
                if not claim(issued):
                    total = issued
                issued += 1
        for w in warps:
            if w["done"]:
                continue
            k = w["k"]
            b = k % nb
            if w["state"] == "wait":
                if k >= tiles and not batch:
                    w["done"] = True
                elif ready[b].test((k // nb) & 1):
                    if in_buf[b] == "end":
                        w["done"] = True
                        continue
                    assert in_buf[b] == k, "a warp reads the wrong tile"
                    if batch and machs[k] != w["mach"]:
                        meet.arrive()
                        w["state"] = "meet1"
                    else:
                        w["state"], w["busy"] = "work", rng.choice([1, 2, 5, 20])
            elif w["state"] == "meet1" and meet.test(w["meet"] & 1):
                w["meet"] += 1
                w["mach"] = machs[k]
                meet.arrive()
                w["state"] = "meet2"
            elif w["state"] == "meet2" and meet.test(w["meet"] & 1):
                w["meet"] += 1
                w["state"], w["busy"] = "work", rng.choice([1, 2, 5, 20])
            elif w["state"] == "work":
                assert in_buf[b] == k, "a buffer was refilled during use"
                w["busy"] -= 1
                if w["busy"] == 0:
                    empty[b].arrive()
                    released[k] = released.get(k, 0) + 1
                    w["k"] += 1
                    w["state"] = "wait"
        if producer_done and all(w["done"] for w in warps):
            assert not inflight, "a copy still in flight at exit"
            return step
    raise AssertionError("deadlock")


def test_single_text_pipeline():
    for nb in (2, 3):
        for tiles in range(0, 24):
            for seed in range(6):
                simulate(tiles, nb=nb, ncw=16, seed=seed)


def test_batch_pipeline_with_machine_changes_and_closing_descriptor():
    for nb in (2, 3):
        for tiles in range(0, 24):
            for seed in range(6):
                rng = random.Random(1000 * nb + 31 * tiles + seed)
                machs = sorted(rng.randint(0, 4) for _ in range(tiles))
                simulate(tiles, machs=machs, nb=nb, ncw=15, seed=seed)
