"""Learned form selector (an extension; the paper picks its methods by
experiment).  A 16 -> 64 -> 64 -> C multilayer perceptron reads the
features of a matrix (spmv_features) and scores C classes, each a way to run
the repeated SpMV: the plain CSR kernel in natural order, or the SB / DB form
or a split at some K with some tile shape.  It is trained on the GPU by the
library's own kernels (spmv_mlp_grad, spmv_mlp_adam) from the autotuner's
timings, and falls back to timing every class when it is unsure.

This module orchestrates those calls; every operation on the network runs in
the library's CUDA kernels."""
import numpy as np

from . import (SPMV_SEL_FEATURES, spmv_features, spmv_mlp_adam, spmv_mlp_fold_scaling,
               spmv_mlp_grad, spmv_mlp_param_count, spmv_mlp_predict, spmv_mlp_work_bytes)

# (framework, K, cta_threads): framework "natural" runs the plain CSR kernel,
# "tiled" the natural order through the tiled kernel
CLASSES = [("natural", 1, 0), ("tiled", 1, 256)] + [
    (fw, K, ct) for fw in ("sb", "db", "split") for K in (16, 256) for ct in (256, 1024)]


def features(m, n, rowptr, colidx):
    return spmv_features(m, n, rowptr, colidx)


class Selector:
    """The network's parameters, its Adam state and the feature scaling."""

    def __init__(self, nc=len(CLASSES), nh=64, seed=0, device="cuda"):
        import torch
        self.nin, self.nh, self.nc = SPMV_SEL_FEATURES, nh, nc
        g = np.random.default_rng(seed)
        # He initialisation of the weights, zero biases
        parts = [g.normal(0, np.sqrt(2.0 / self.nin), (nh, self.nin)), np.zeros(nh),
                 g.normal(0, np.sqrt(2.0 / nh), (nh, nh)), np.zeros(nh),
                 g.normal(0, np.sqrt(1.0 / nh), (nc, nh)), np.zeros(nc)]
        flat = np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)
        assert flat.size == spmv_mlp_param_count(self.nin, nh, nc)
        self.params = torch.from_numpy(flat).to(device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self.device = device

    def _x(self, F):
        import torch
        X = np.ascontiguousarray(np.atleast_2d(F), dtype=np.float32)
        return torch.from_numpy(X).to(self.device)

    def fit(self, F, labels, epochs=300, lr=3e-3, batch=64, seed=0):
        """Train on features F (N x 16) and class labels (N); returns the
        loss of each epoch (full passes over shuffled mini-batches)."""
        import torch
        F = np.asarray(F, dtype=np.float32)
        # training reads standardised features; afterwards the scaling is
        # folded into the first layer, so that the network reads raw ones
        mu = F.mean(axis=0).astype(np.float32)
        sd = (F.std(axis=0) + 1e-6).astype(np.float32)
        X = self._x((F - mu) / sd)
        y = torch.from_numpy(np.asarray(labels, dtype=np.int32)).to(self.device)
        grads = torch.empty_like(self.params)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        work = torch.empty(spmv_mlp_work_bytes(self.nh, self.nc, batch), dtype=torch.uint8,
                           device=self.device)
        rng = np.random.default_rng(seed)
        hist = []
        n = X.shape[0]
        for _ in range(epochs):
            order = torch.from_numpy(rng.permutation(n)).to(self.device)
            tot = 0.0
            for s in range(0, n, batch):
                idx = order[s:s + batch]
                xb, yb = X[idx].contiguous(), y[idx].contiguous()
                spmv_mlp_grad(self.params, self.nin, self.nh, self.nc, xb, yb, grads, loss, work)
                self.step += 1
                spmv_mlp_adam(self.params, self.nin, self.nh, self.nc, grads, self.m, self.v,
                              self.step, lr)
                tot += float(loss.item()) * idx.numel()
            hist.append(tot / n)
        spmv_mlp_fold_scaling(self.params, self.nin, self.nh, self.nc,
                              torch.from_numpy(mu).to(self.device),
                              torch.from_numpy(sd).to(self.device))
        return hist

    def predict(self, F):
        """(class, softmax probability of that class) per row of raw
        features F, from the library's kernels."""
        import torch
        X = self._x(F)
        cls = torch.empty(X.shape[0], dtype=torch.int32, device=self.device)
        conf = torch.empty(X.shape[0], dtype=torch.float32, device=self.device)
        work = torch.empty(spmv_mlp_work_bytes(self.nh, self.nc, X.shape[0]), dtype=torch.uint8,
                           device=self.device)
        spmv_mlp_predict(self.params, self.nin, self.nh, self.nc, X, cls, conf, work)
        return cls.cpu().numpy(), conf.cpu().numpy()

    def choose(self, F, min_confidence=0.0):
        """Class index per matrix, or -1 where the top probability is below
        min_confidence (the caller then times every class)."""
        cls, conf = self.predict(F)
        return np.where(conf >= min_confidence, cls, -1)
