"""Host logic of the Python binding, on the CPU with a stand-in for libdl: the order in which
contexts and programs are freed.  A program's destruction locks its context, so closing a
context must first close the programs still alive on it, and a program whose context is gone
must not call into the library again."""
import gc

from paper_1608_00139_gb300 import dl


class FakeLib:
    """Records the C calls the binding makes; handles are plain integers."""

    def __init__(self):
        self.calls = []
        self.live_ctx = set()
        self.live_prog = {}

    def dl_create(self, out, device, cfg):
        h = 1000 + len(self.calls)
        out._obj.value = h
        self.live_ctx.add(h)
        self.calls.append(("create", h))
        return dl.DL_OK

    def dl_destroy(self, h):
        h = h.value
        assert h in self.live_ctx
        assert all(c != h for c in self.live_prog.values()), "a program outlives its context"
        self.live_ctx.discard(h)
        self.calls.append(("destroy", h))
        return dl.DL_OK

    def dl_program_create(self, ctx, text, out):
        h = 5000 + len(self.calls)
        out._obj.value = h
        self.live_prog[h] = ctx.value
        self.calls.append(("program_create", h))
        return dl.DL_OK

    def dl_program_destroy(self, h):
        h = h.value
        assert self.live_prog.pop(h) in self.live_ctx, "program destroyed after its context"
        self.calls.append(("program_destroy", h))
        return dl.DL_OK

    def dl_last_error(self):
        return b""


def with_fake(monkeypatch):
    fake = FakeLib()
    monkeypatch.setattr(dl, "lib", lambda: fake)
    return fake


def test_closing_a_context_closes_its_programs_first(monkeypatch):
    fake = with_fake(monkeypatch)
    c = dl.Context(0)
    progs = [c.program("r(X,Y) :- e(X,Y).") for _ in range(3)]
    progs[1].close()
    c.close()
    kinds = [k for k, _ in fake.calls]
    assert kinds[-1] == "destroy"
    assert kinds.count("program_destroy") == 3 and not fake.live_prog
    assert all(p._h is None for p in progs)
    n = len(fake.calls)
    for p in progs:  # no call into the library once the context is gone
        p.close()
    del progs
    gc.collect()
    assert len(fake.calls) == n


def test_a_program_kept_alive_by_a_reference_cycle(monkeypatch):
    """The case that freed a context under a live program: an exception info object (a
    reference cycle through the frame) keeps the program until a garbage collection that may
    come after the context's explicit close."""
    fake = with_fake(monkeypatch)
    c = dl.Context(0)

    def holder():
        prog = c.program("r(X,Y) :- e(X,Y).")
        try:
            raise ValueError
        except ValueError as err:
            keep = err  # frame -> err -> traceback -> frame
        return keep

    cyc = holder()
    c.close()  # the program is still alive through the cycle
    del cyc
    gc.collect()
    assert not fake.live_prog and not fake.live_ctx


def test_programs_on_separate_contexts(monkeypatch):
    fake = with_fake(monkeypatch)
    a, b = dl.Context(0), dl.Context(0)
    pa, pb = a.program("r(X,Y) :- e(X,Y)."), b.program("r(X,Y) :- e(X,Y).")
    a.close()
    assert pa._h is None and pb._h is not None
    pb.close()
    b.close()
    assert not fake.live_prog and not fake.live_ctx
