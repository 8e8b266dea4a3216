"""Training driver of the learned exit proposal (argument marshalling around the
C-ABI; data generation, the network's forward and backward passes and the
optimiser all run in the library's kernels).

A proposal is trained for one target grid (cell size, frequency bins,
temperature): uniform media at L density levels, each a 3^3 grid of the
target's cell size whose centre cell carries the interior rows of a uniform
brick, produce first passages through a b^3 brick from a cell of the brick
(folded into the fundamental domain of the cube's symmetry group) at a bin of
the positive-frequency side whose cell optical depth lies in [tau_lo, tau_hi].
A static uniform brick is symmetric under x -> -x and under the cube's
reflections and axis permutations, so a packet at negative frequency is
mirrored, and its cell folded, at inference.  The walk is Markov in
(cell, bin): a packet can be handed to the proposal in any state it serves.

The network has three heads: exit face x exit bin (A), log2 step bucket (B)
and, per exit face, the exit cell on that face (C).
"""
from __future__ import annotations

import numpy as np

from . import rddmc as R
from . import workloads as W

N_STEP_BUCKETS = 32


class ExitProposal:
    def __init__(self, target: W.Workload, brick: int, rho_levels, tau_lo=5.0, tau_hi=200.0, device="cuda",
                 hidden_seed=0x5EED0601, position_head=True):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.target = target
        self.b = int(brick)
        self.J = target.J
        dz = 2.0 * target.R / target.n[0]
        self.dz = dz
        R3 = 1.5 * dz
        self.levels = []
        self.problems = []
        lk, jlo, jhi = [], [], []
        lp = None
        for rho in rho_levels:
            tau3 = target.tau0 / target.R * float(rho) * R3
            w = W.Workload(f"level_{rho:.4g}", 3, (3, 3, 3), target.J, target.x_min, target.x_max, tau3, target.T,
                           1, 1, R=R3)
            p = R.Problem(w, device=self.device)
            tau = R.cell_tau(p.grid, p.table.data_ptr(), 13, self.J, p.stream()).astype(np.float64)
            kdz = 2.0 * tau3 / 3.0  # k0 dz of the level
            if lp is None:
                lp = np.log10(np.maximum(tau, 1e-300)) - np.log10(kdz)
            xc = 0.5 * (w.edges()[1:] + w.edges()[:-1])
            ok = np.nonzero((xc >= 0) & (tau >= tau_lo) & (tau <= tau_hi))[0]
            if ok.size == 0:
                continue
            # a contiguous run on the positive side (the wing, where tau falls with |x|)
            lo, hi = int(ok.min()), int(ok.max())
            if not np.all((tau[lo:hi + 1] >= tau_lo) & (tau[lo:hi + 1] <= tau_hi)):
                continue
            self.levels.append(float(rho))
            self.problems.append(p)
            lk.append(np.log10(kdz))
            jlo.append(lo)
            jhi.append(hi)
        if not self.problems:
            raise ValueError("no density level has bins in the requested optical-depth range")
        self.jlo, self.jhi = np.array(jlo, np.int32), np.array(jhi, np.int32)
        t = lambda a, dt: torch.as_tensor(np.asarray(a), dtype=dt, device=self.device)
        self.lk = t(np.array(lk, np.float32), torch.float32)
        self.lp = t(lp.astype(np.float32), torch.float32)
        self.xc = t((0.5 * (target.edges()[1:] + target.edges()[:-1])).astype(np.float32), torch.float32)
        self.nA = 6 * self.J
        self.nB = N_STEP_BUCKETS
        self.S = self.b * self.b
        self.nC = 6 * self.S if position_head else 0
        self.n_out = ((self.nA + self.nB + self.nC + 15) // 16) * 16
        n_par = R.mlp_param_count(self.n_out)
        rng = np.random.default_rng(hidden_seed)
        flat = []
        for (o, i) in [(128, 16), (128, 128), (128, 128), (self.n_out, 128)]:
            flat.append(rng.normal(0.0, np.sqrt(2.0 / i), o * i))   # He initialisation
            flat.append(np.zeros(o))
        flat = np.concatenate(flat).astype(np.float32)
        assert flat.size == n_par
        self.wf = t(flat, torch.float32)
        self.wb = torch.empty(n_par, dtype=torch.bfloat16, device=self.device)
        R.mlp_to_bf16(self.n_out, self.wf.data_ptr(), self.wb.data_ptr(), self.stream())
        self.m = torch.zeros_like(self.wf)
        self.v = torch.zeros_like(self.wf)
        self.grad = torch.zeros_like(self.wf)
        self.step = 0

    def stream(self) -> int:
        return self.torch.cuda.current_stream(self.device).cuda_stream

    # ------------------------------------------------------------------ data
    def generate(self, n: int, seed: int, p0: int = 0, cap: int = 10_000_000) -> dict:
        """n first-passage samples with network inputs and targets (device tensors)."""
        torch = self.torch
        out = torch.empty(8 * n, dtype=torch.int32, device=self.device)
        steps = torch.empty(n, dtype=torch.int64, device=self.device)
        X = torch.empty((n, 16), dtype=torch.bfloat16, device=self.device)
        tA = torch.empty(n, dtype=torch.int32, device=self.device)
        tB = torch.empty(n, dtype=torch.int32, device=self.device)
        tC = torch.empty(n, dtype=torch.int32, device=self.device)
        tr = R.FpTrain(X.data_ptr(), tA.data_ptr(), tB.data_ptr(), self.lk.data_ptr(), self.lp.data_ptr(),
                       self.xc.data_ptr(), tC.data_ptr())
        R.fp_generate([p.grid for p in self.problems], [p.table.data_ptr() for p in self.problems], self.b, self.jlo,
                      self.jhi, seed, p0, n, cap, out.data_ptr(), steps.data_ptr(), tr, self.stream())
        return dict(X=X, tA=tA, tB=tB, tC=tC, rec=out.view(n, 8), steps=steps)

    # ------------------------------------------------------------------ training
    def _loss_grad(self, X, tA, tB, tC, B, work, loss):
        R.mlp_loss_grad(self.n_out, self.nA, self.nB, self.wf.data_ptr(), self.wb.data_ptr(), X.data_ptr(),
                        tA.data_ptr(), tB.data_ptr(), B, work.data_ptr(), self.grad.data_ptr(), loss.data_ptr(),
                        self.stream(), nC=self.nC, S=self.S, d_tc=tC.data_ptr() if self.nC else 0)

    def loss_grad(self, X, tA, tB, tC=None):
        B = X.shape[0]
        work = self.torch.empty(R.mlp_work_bytes(B, self.n_out), dtype=self.torch.uint8, device=self.device)
        loss = self.torch.zeros(1, dtype=self.torch.float32, device=self.device)
        if tC is None:
            tC = self.torch.full((B,), -1, dtype=self.torch.int32, device=self.device)
        self._loss_grad(X, tA, tB, tC, B, work, loss)
        return loss

    def train(self, data: dict, iters: int, batch: int = 8192, lr: float = 1e-3, seed: int = 1, log_every=0,
              lr_final: float = None):
        """Adam on random minibatches; the step size decays from lr to lr_final
        (default lr / 20) on a cosine schedule."""
        torch = self.torch
        lr_final = lr / 20.0 if lr_final is None else lr_final
        n = data["X"].shape[0]
        gen = torch.Generator(device=self.device)
        gen.manual_seed(seed)
        work = torch.empty(R.mlp_work_bytes(batch, self.n_out), dtype=torch.uint8, device=self.device)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        hist = []
        for it in range(iters):
            idx = torch.randint(0, n, (batch,), device=self.device, generator=gen)
            X, tA, tB, tC = (data[k][idx].contiguous() for k in ("X", "tA", "tB", "tC"))
            self._loss_grad(X, tA, tB, tC, batch, work, loss)
            self.step += 1
            lr_t = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * it / max(1, iters - 1)))
            R.mlp_adam(self.n_out, self.wf.data_ptr(), self.wb.data_ptr(), self.grad.data_ptr(), self.m.data_ptr(),
                       self.v.data_ptr(), self.step, lr_t, stream=self.stream())
            if log_every and (it % log_every == 0 or it == iters - 1):
                hist.append((it, float(loss.item()) / batch))
        return hist

    def mean_loss(self, data: dict, batch: int = 8192) -> float:
        n = (data["X"].shape[0] // batch) * batch
        tot = 0.0
        for s in range(0, n, batch):
            sl = slice(s, s + batch)
            tot += float(self.loss_grad(*(data[k][sl].contiguous() for k in ("X", "tA", "tB", "tC"))).item())
        return tot / n

    def logits(self, X):
        B = X.shape[0]
        work = self.torch.empty(R.mlp_work_bytes(B, self.n_out), dtype=self.torch.uint8, device=self.device)
        out = self.torch.empty((B, self.n_out), dtype=self.torch.float32, device=self.device)
        R.mlp_forward(self.n_out, self.wf.data_ptr(), self.wb.data_ptr(), X.data_ptr(), B, work.data_ptr(),
                      out.data_ptr(), self.stream())
        return out

    # ------------------------------------------------------------------ walking with the proposal
    def attach(self, problem, brick_rho, offset: int = 0, batch: int = 4096, margin: int = 0,
               exclude_surface: bool = False):
        """Proposal state for walking `problem`, its grid cut into bricks of
        (self.b + 2 margin)^3 cells with boundaries at cell indices = offset
        (mod that size) and per-brick density brick_rho (partial bricks
        included, brick index axis 0 fastest); each brick serves its inner cube
        of self.b^3 cells.  Bricks whose density lies outside the trained levels
        take no proposals; nor do partial bricks, nor (exclude_surface) bricks
        on the lattice's outer layer.  With margin >= 1 on a brick-uniform
        medium the served cubes see only their own medium and no surface
        exclusion is needed."""
        torch = self.torch
        lat = self.b + 2 * int(margin)
        rho = np.asarray(brick_rho, dtype=np.float64)
        lk = np.log10(problem.w.tau0 / problem.w.R * rho * self.dz)
        lo, hi = np.log10(min(self.levels)), np.log10(max(self.levels))
        ok = (np.log10(rho) >= lo) & (np.log10(rho) <= hi)
        if exclude_surface:
            nb = [(problem.w.n[a] + (lat - offset % lat) % lat + lat - 1) // lat for a in range(3)]
            c2, c1, c0 = np.meshgrid(np.arange(nb[2]), np.arange(nb[1]), np.arange(nb[0]), indexing="ij")
            inner = np.ones_like(c0, dtype=bool)
            for c, m in ((c0, nb[0]), (c1, nb[1]), (c2, nb[2])):
                inner &= (c > 0) & (c < m - 1)
            ok &= inner.reshape(-1)
        lk = np.where(ok, lk, -1.0e30).astype(np.float32)
        return dict(
            lk=torch.as_tensor(lk, device=self.device),
            count=torch.zeros(1, dtype=torch.int64, device=self.device),
            offset=int(offset), lattice=lat, margin=int(margin),
            batch=batch,
            work=torch.empty(R.mlp_work_bytes(batch, self.n_out) + 256 + batch * 32 + 256 + batch * self.n_out * 4
                             + 4096, dtype=torch.uint8, device=self.device))

    def proposal(self, att, qpid, tau_lo: float, tau_hi: float):
        """The C-ABI proposal struct for an attach() state and a queue buffer."""
        return R.Proposal(att["lattice"], att["offset"], att["lk"].data_ptr(), self.lp.data_ptr(), self.xc.data_ptr(),
                          np.log10(tau_lo), np.log10(tau_hi), att["count"].data_ptr(), qpid.data_ptr(),
                          int(att["lk"].numel()), att["margin"])

    def run(self, problem, brick_rho, n_packets: int, seed: int, offset: int = 0, steps_per_launch: int = 0,
            batch: int = 65536, tau_lo: float = 5.0, tau_hi: float = 200.0, max_epochs: int = 1_000_000,
            margin: int = 0, exclude_surface: bool = False, time_slice_us: int = 1000) -> dict:
        """Walk n_packets on `problem` with proposals: walk launches bounded by
        time_slice_us of wall time (and steps_per_launch transitions per packet,
        0 = no bound) alternate with proposal rounds for the packets parked
        meanwhile, until every packet has escaped or been aborted.  The tallies
        do not depend on the slicing.  Returns the tallies and the number of
        walk launches, proposal rounds and proposals served."""
        torch = self.torch
        problem.ensure_state(n_packets)
        att = self.attach(problem, brick_rho, offset, batch, margin, exclude_surface)
        qpid = torch.empty(n_packets, dtype=torch.int64, device=self.device)
        prop = self.proposal(att, qpid, tau_lo, tau_hi)
        problem.reset()
        launches = rounds = served = 0
        t = None
        for ep in range(max_epochs):
            problem.launch(n_packets, seed, steps_per_launch=steps_per_launch, resume=1 if ep else 0, proposal=prop,
                           time_slice_us=time_slice_us)
            launches += 1
            k = R.propose(problem.grid, problem.table.data_ptr(), prop, seed, n_packets, problem.state.data_ptr(),
                          problem.tally.data_ptr(), self.n_out, self.nA, self.nB, self.wf.data_ptr(),
                          self.wb.data_ptr(), batch, att["work"].data_ptr(), problem.stream(), nC=self.nC)
            served += k
            rounds += 1 if k else 0
            # the termination test synchronises: every few epochs, and whenever a
            # round found nothing parked (the end is near or reached)
            if k == 0 or ep % 8 == 7:
                t = problem.read()
                if t["escaped"] + t["aborted"] >= n_packets:
                    break
        t = problem.read()
        t["launches"], t["rounds"], t["served"] = launches, rounds, served
        return t
