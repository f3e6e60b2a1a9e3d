"""Host model of the barrier protocol of the expansion kernel's dual-issuer form (form 5): one
producer fills a ring of NL stages in sequence (one stage per sub-stage: one per term of a full
item, one per plane of a packed tail item), and two stage-2 warps take alternate terms.

An mbarrier wait names only the parity of the phase it waits for, so a wait is correct only
while the barrier is at most one phase behind the waiter: with c phases completed, a waiter for
fill n (parity n & 1) must find c in {n, n + 1}.  c = n - 1 would pass at once (the parity of
an older phase matches), c = n + 2 would wait forever.  With a single consumer this holds by
construction; with two consumers a warp can reach a stage whose previous fill belongs to the
other warp's term that has not been waited on yet.  The kernel orders the waits with a token:
a warp waits for the stages of term g only after the other warp has seen all stages of term
g - 1 arrive.  Random schedules check that the token keeps every wait within one phase, and
that without it some schedule breaks the rule."""
import random

import pytest


class Barrier:
    def __init__(self):
        self.completed = 0          # phases completed


def simulate(rng, items, NL, use_token):
    """One random schedule; returns the first violation found (or None).  items: list of sub-stage
    counts per term, in the CTA's term order."""
    Q = sum(items)
    first_q = []                     # first sub-stage index of each term
    q = 0
    for n in items:
        first_q.append(q)
        q += n
    full = [Barrier() for _ in range(NL)]
    empty = [Barrier() for _ in range(NL)]
    tok = [Barrier(), Barrier()]
    pending = []                     # asynchronous completions: (barrier,)
    prod_q = 0                       # next sub-stage the producer fills
    # consumer state: term index (own parity), sub-stage within it, phase of its action
    cons = [dict(g=0, sp=0, token_ok=False), dict(g=1, sp=0, token_ok=False)]

    def check(bar, n, who):
        c = bar.completed
        if c not in (n, n + 1):
            return f"{who}: waits for fill {n} but {c} phases are complete"
        return None

    steps = 0
    while steps < 100000:
        steps += 1
        actions = []
        if prod_q < Q:
            actions.append("prod")
        for w in (0, 1):
            if cons[w]["g"] < len(items):
                actions.append(w)
        if pending:
            actions.append("async")
        if not actions:
            return None
        a = rng.choice(actions)
        if a == "async":
            bar = pending.pop(rng.randrange(len(pending)))
            bar.completed += 1
        elif a == "prod":
            s, n = prod_q % NL, prod_q // NL
            if n > 0:                # wait for the consumption of fill n - 1 of this stage
                err = check(empty[s], n - 1, "producer")
                if err:
                    return err
                if (empty[s].completed & 1) == ((n - 1) & 1):
                    continue         # not yet
            pending.append(full[s])  # the copies land later
            prod_q += 1
        else:
            st = cons[a]
            g = st["g"]
            if use_token and g > 0 and not st["token_ok"]:
                n = (g - 1) >> 1     # the other warp's token for term g - 1
                if (tok[(g - 1) & 1].completed & 1) == (n & 1):
                    continue
                st["token_ok"] = True
            qq = first_q[g] + st["sp"]
            s, n = qq % NL, qq // NL
            err = check(full[s], n, f"warp {a}, term {g}")
            if err:
                return err
            if (full[s].completed & 1) == (n & 1):
                continue             # stage not landed yet
            pending.append(empty[s])  # the MMAs release the stage when they have run
            st["sp"] += 1
            if st["sp"] == items[g]:
                if use_token:
                    tok[g & 1].completed += 1   # all stages of term g seen: pass the token
                st["g"] += 2
                st["sp"] = 0
                st["token_ok"] = False
    return "schedule did not finish"


def item_mix(rng, terms, tailp):
    """Terms of full items (one sub-stage) and packed tail items (tailp sub-stages), in runs of
    T terms per item as the kernel walks them."""
    out = []
    T = rng.choice([2, 3, 5, 6])
    while len(out) < terms:
        n = tailp if rng.random() < 0.3 else 1
        out.extend([n] * T)
    return out[:terms]


@pytest.mark.parametrize("NL,tailp", [(4, 4), (4, 2), (3, 4), (4, 5), (2, 3)])
def test_token_keeps_every_wait_within_one_phase(NL, tailp):
    rng = random.Random(1000 * NL + tailp)
    for _ in range(300):
        items = item_mix(rng, 40, tailp)
        err = simulate(rng, items, NL, use_token=True)
        assert err is None, err


def test_without_the_token_some_schedule_breaks_the_rule():
    rng = random.Random(7)
    found = None
    for _ in range(2000):
        items = item_mix(rng, 40, 4)
        found = simulate(rng, items, 4, use_token=False)
        if found and "phases are complete" in found:
            break
    assert found and "phases are complete" in found
