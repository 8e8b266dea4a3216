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


# ----------------------------------------------------------------------------- media that vary cell by cell
F_MU = 0.5  # angle factor of the comoving shift across a face (eq. velocity-shift)


def region_summaries(w: W.Workload, n_rel, v_kms, brick: int, margin: int, offset: int = 0):
    """Per lattice brick (axis 0 fastest, partial bricks included) the 8
    floats of rddmc_fp_region.d_summary for its inner cube (side brick - 2
    margin), and whether the brick lies wholly inside the grid.  Host-side
    description of the medium: no step of the walk."""
    n = w.n[0]
    assert w.ndim == 3 and w.n[1] == n and w.n[2] == n
    nbx, cidx, sh = W.brick_lattice(n, brick, offset)
    r = brick - 2 * margin
    dz = 2.0 * w.R / n
    vth = 12.85 * np.sqrt(w.T / 1.0e4)
    lg = np.log10(np.asarray(n_rel, dtype=np.float64)).reshape(n, n, n)       # [i2, i1, i0]
    v = (np.zeros((n, n, n, 3)) if v_kms is None else np.asarray(v_kms, dtype=np.float64).reshape(n, n, n, 3))
    u = (2.0 * np.arange(r) + 1.0) / r - 1.0
    out = np.zeros((nbx ** 3, 8), dtype=np.float32)
    full = np.zeros(nbx ** 3, dtype=bool)
    lk0 = np.log10(w.tau0 / w.R * dz)
    for b2 in range(nbx):
        for b1 in range(nbx):
            for b0 in range(nbx):
                bi = b0 + nbx * (b1 + nbx * b2)
                lo = [bb * brick - sh for bb in (b0, b1, b2)]
                if min(lo) < 0 or max(lo) + brick > n:
                    continue
                full[bi] = True
                s = [slice(lo[a] + margin, lo[a] + margin + r) for a in (2, 1, 0)]  # [i2, i1, i0]
                y = lg[s[0], s[1], s[2]]
                mu = y.mean()
                out[bi, 0] = lk0 + mu
                out[bi, 1] = y.std()
                dy = y - mu
                den = (u * u).sum() * r * r
                out[bi, 2] = (dy * u[None, None, :]).sum() / den   # axis 0 (x): last array index
                out[bi, 3] = (dy * u[None, :, None]).sum() / den
                out[bi, 4] = (dy * u[:, None, None]).sum() / den
                vv = v[s[0], s[1], s[2]]
                d = [F_MU * (vv[:, :, :-1, 0] - vv[:, :, 1:, 0]) / vth,
                     F_MU * (vv[:, :-1, :, 1] - vv[:, 1:, :, 1]) / vth,
                     F_MU * (vv[:-1, :, :, 2] - vv[1:, :, :, 2]) / vth]
                d = np.concatenate([x.ravel() for x in d])
                out[bi, 5] = d.mean() if d.size else 0.0
                out[bi, 6] = np.sqrt((d * d).mean()) if d.size else 0.0
    return out, full


class RegionProposal(ExitProposal):
    """The learned exit proposal for a medium that varies from cell to cell.

    Regions are the inner cubes (side r = brick - 2 margin) of a brick lattice
    over the target grid.  First passages are generated on the target's own
    table (rddmc_fp_region_generate: the walk's transitions, Doppler rebins
    included), and the network is conditioned on a summary of the region
    (its mean density and spread, density slopes, mean and rms Doppler shift
    per crossing), the start cell's density, position and bin, in the world
    frame.  The proposal is an approximation of the region's exact exit law;
    the plain walk judges its escape spectrum."""

    def __init__(self, problem, n_rel, v_kms, brick: int, margin: int, offset: int = 0, tau_lo=5.0, tau_hi=1.0e12,
                 hidden_seed=0x5EED0611):
        import torch
        self.torch = torch
        self.device = problem.device
        self.problem = problem
        w = problem.w
        self.target = w
        self.J = w.J
        self.lattice, self.margin, self.offset = int(brick), int(margin), int(offset)
        self.b = self.lattice - 2 * self.margin           # the region's side
        self.dz = 2.0 * w.R / w.n[0]
        self.tau_lo, self.tau_hi = float(tau_lo), float(tau_hi)
        summ, full = region_summaries(w, n_rel, v_kms, self.lattice, self.margin, self.offset)
        self.summary_np, self.full = summ, full
        # log10 of the bin-mean profile phi_j from the target's own rows (any cell)
        tau = R.cell_tau(problem.grid, problem.table.data_ptr(), 0, self.J, problem.stream()).astype(np.float64)
        nrel0 = float(np.asarray(n_rel).reshape(-1)[0])
        lp = (np.log10(np.maximum(tau, 1e-300)) - np.log10(w.tau0 / w.R * nrel0 * self.dz)).astype(np.float32)
        # eligible states, decided in FP32 exactly as the walk decides them
        llo, lhi = np.float32(np.log10(self.tau_lo)), np.float32(np.log10(self.tau_hi))
        bricks, off, bins = [], [0], []
        for bi in np.nonzero(full)[0]:
            l = np.float32(summ[bi, 0]) + lp
            ok = np.nonzero((l >= llo) & (l <= lhi))[0]
            if ok.size:
                bricks.append(int(bi))
                bins.extend(int(j) for j in ok)
                off.append(len(bins))
        if not bricks:
            raise ValueError("no brick has bins in the requested optical-depth range")
        lk = np.full(len(full), -1.0e30, dtype=np.float32)
        lk[bricks] = summ[bricks, 0]
        t = lambda a, dt: torch.as_tensor(np.asarray(a), dtype=dt, device=self.device)
        self.bricks = t(np.array(bricks, np.int32), torch.int32)
        self.bin_off = t(np.array(off, np.int32), torch.int32)
        self.bins = t(np.array(bins, np.int32), torch.int32)
        self.summary = t(summ.reshape(-1), torch.float32)
        self.brick_lk = t(lk, torch.float32)
        self.lp = t(lp, torch.float32)
        self.lk = t(np.zeros(1, np.float32), torch.float32)  # unused in region mode
        self.xc = t((0.5 * (w.edges()[1:] + w.edges()[:-1])).astype(np.float32), torch.float32)
        self.levels = []
        self.nA = 6 * self.J
        self.nB = N_STEP_BUCKETS
        self.S = self.b * self.b
        self.nC = 6 * self.S
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

    def region_struct(self):
        return R.FpRegion(self.lattice, self.offset, self.margin, int(self.bricks.numel()), self.bricks.data_ptr(),
                          self.bin_off.data_ptr(), self.bins.data_ptr(), self.summary.data_ptr())

    def generate(self, n: int, seed: int, p0: int = 0, cap: int = 10_000_000) -> dict:
        """n first passages out of the target's regions with network inputs and targets (device tensors)."""
        torch = self.torch
        out = torch.empty(8 * n, dtype=torch.int32, device=self.device)
        steps = torch.empty(n, dtype=torch.int64, device=self.device)
        X = torch.empty((n, 16), dtype=torch.bfloat16, device=self.device)
        tA = torch.empty(n, dtype=torch.int32, device=self.device)
        tB = torch.empty(n, dtype=torch.int32, device=self.device)
        tC = torch.empty(n, dtype=torch.int32, device=self.device)
        tr = R.FpTrain(X.data_ptr(), tA.data_ptr(), tB.data_ptr(), self.lk.data_ptr(), self.lp.data_ptr(),
                       self.xc.data_ptr(), tC.data_ptr())
        R.fp_region_generate(self.problem.grid, self.problem.table.data_ptr(), self.region_struct(), seed, p0, n, cap,
                             out.data_ptr(), steps.data_ptr(), tr, self.stream())
        return dict(X=X, tA=tA, tB=tB, tC=tC, rec=out.view(n, 8), steps=steps)

    def attach(self, problem, brick_rho=None, offset: int = 0, batch: int = 4096, margin: int = 0,
               exclude_surface: bool = False):
        """Proposal state for walking the target (the lattice and margin are the
        proposal's own; brick_rho, offset and margin arguments are ignored)."""
        torch = self.torch
        return dict(
            lk=self.brick_lk, count=torch.zeros(1, dtype=torch.int64, device=self.device),
            offset=self.offset, lattice=self.lattice, margin=self.margin, batch=batch,
            work=torch.empty(R.mlp_work_bytes(batch, self.n_out) + 256 + batch * 32 + 256 + batch * self.n_out * 4
                             + 4096, dtype=torch.uint8, device=self.device))

    def proposal(self, att, qpid, tau_lo: float, tau_hi: float):
        return R.Proposal(att["lattice"], att["offset"], att["lk"].data_ptr(), self.lp.data_ptr(), self.xc.data_ptr(),
                          np.log10(tau_lo), np.log10(tau_hi), att["count"].data_ptr(), qpid.data_ptr(),
                          int(att["lk"].numel()), att["margin"], self.summary.data_ptr())

    def run(self, problem=None, brick_rho=None, n_packets: int = 0, seed: int = 0, **kw) -> dict:
        """Walk n_packets on the target with proposals (see ExitProposal.run);
        the eligibility band is the proposal's own tau_lo, tau_hi."""
        kw.setdefault("tau_lo", self.tau_lo)
        kw.setdefault("tau_hi", self.tau_hi)
        return ExitProposal.run(self, self.problem if problem is None else problem, None, n_packets, seed, **kw)
