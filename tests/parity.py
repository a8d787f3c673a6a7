"""Helpers shared by the GPU parity tests: the pass simulator's counters
against a render's per-pass records, and the oracle's pixel records with
ambiguous pixels resolved by the GPU's (validated) answer."""
import numpy as np


def resolved_pix(sc, fb):
    """The oracle's per-pixel records with every ambiguous pixel (where a
    correct single-precision renderer may pick either of two answers) set to
    the GPU's answer after checking that the answer is a valid one: a hit in
    one of the ray's visible blocks (in its full visible list), or a miss.
    The pass simulator run on these records is then exact for the whole
    image, so its counters are compared unconditionally."""
    pix = sc.pix.copy()
    amb = np.nonzero(pix["amb"] != 0)[0]
    for p in amb:
        lst = sc.vis[sc.off[p]:sc.off[p] + pix["n_visible"][p]]
        if fb["status"][p] == 1:
            where = np.nonzero(lst == fb["block"][p])[0]
            assert where.size == 1, "pixel %d hit block %d outside its visible list" % (p, fb["block"][p])
            pix["hit"][p] = 1
            pix["hit_index"][p] = int(where[0])
        else:
            assert fb["status"][p] == 2, p
            pix["hit"][p] = 0
            pix["hit_index"][p] = -1
    return pix


def check_counters(st, passes):
    assert len(st) == len(passes)
    for s, p in zip(st, passes):
        for name in ("n_active", "k", "k_used", "n_processed", "retries", "n_entries", "n_visible",
                     "n_requested", "n_decoded", "n_evicted", "n_term_hit", "n_term_miss"):
            assert int(s[name]) == int(p[name]), (name, s["pass"], int(s[name]), int(p[name]))


