"""Host-side restatement of the surrogate advance loop, for the tests only.

It drives the same library primitives one by one from Python (snapshot, the network's forward
through the trainer, restart from a snapshot, solver steps, snapshot comparison, state copies) in
the order that vlb_surrogate_advance documents, so that the library's loop can be checked against it
window by window and bit for bit.  Windows are always eager here (no graph)."""
import math

from paper_1904_10070_gb300 import vlb


class ReferenceAdvancer:
    def __init__(self, trainer, solver, window=50, check_every=4, phi_tol=1e-2, norm="l2"):
        import torch
        self.tr, self.s, self.window = trainer, solver, window
        self.check_every, self.phi_tol, self.norm = check_every, phi_tol, norm
        self.R = solver.p.R / solver.p.r
        self.stream = solver.stream
        N = solver.p.n_theta * solver.p.n_phi
        with torch.cuda.stream(self.stream):
            self.snap = torch.empty((N, 4), dtype=torch.float32, device="cuda")
            self.pred = torch.empty_like(self.snap)
            self.check = torch.empty_like(self.snap)
            self.norm8 = torch.empty(8, dtype=torch.float32, device="cuda")
            self.cmp = torch.empty(4, dtype=torch.float64, device="cuda")
            self.work = torch.empty(vlb.vlb_reduce_workspace_bytes(), dtype=torch.uint8, device="cuda")
            ptr, stride = vlb.vlb_state_device(solver.h)
            off = ptr - solver.workspace.data_ptr()
            self.state = solver.workspace[off:off + 18 * stride * 4]
            self.good = torch.empty_like(self.state)
        t = solver.totals()
        self.conserve = (t[0], t[1])
        self.solver_only = self.since_good = self.count = 0
        self.kinds, self.errors = [], []

    def _save(self):
        self.good.copy_(self.state)
        self.since_good = 0

    def window_step(self):
        import torch
        with torch.cuda.stream(self.stream):
            return self._window_step()

    def _window_step(self):
        s, w = self.s, self.window
        if self.count == 0:
            self._save()
        self.count += 1
        e2 = einf = math.nan
        if self.solver_only > 0:
            s.step(w)
            self.solver_only -= 1
            self.since_good += 1
            if self.solver_only == 0:
                self._save()
            kind = "solver"
        elif self.check_every > 0 and self.count % self.check_every == 0:
            vlb.vlb_get_snapshot(s.h, self.snap)
            self.tr.predict(self.snap, self.R, self.norm8, self.pred)
            s.step(w)
            vlb.vlb_get_snapshot(s.h, self.check)
            vlb.vlb_snapshot_compare(self.pred.shape[0], self.pred, self.check, self.work, self.cmp,
                                     self.stream.cuda_stream)
            dmax, bmax, d2, b2 = (float(x) for x in self.cmp.cpu())
            einf = dmax / bmax if bmax > 0 else math.inf
            e2 = math.sqrt(d2 / b2) if b2 > 0 else math.inf
            err = e2 if self.norm == "l2" else einf
            if err <= self.phi_tol:
                self._save()
                kind = "checked"
            else:
                self.state.copy_(self.good)
                s.step(w * (self.since_good + 1))
                self.solver_only = self.check_every
                self._save()
                kind = "fallback"
        else:
            vlb.vlb_get_snapshot(s.h, self.snap)
            self.tr.predict(self.snap, self.R, self.norm8, self.pred)
            vlb.vlb_set_snapshot(s.h, self.pred, self.conserve, keep_neq=True)
            self.since_good += 1
            kind = "surrogate"
        self.kinds.append(kind)
        self.errors.append((e2, einf))
        return kind

    def advance(self, nwin):
        return [self.window_step() for _ in range(nwin)]
