"""Training the tuner network on a user's own fields.

Labels come from the sampled tuner (Sec. 6): for each training field and
relative bound, the sampled tuner's level-1 interpolator and dimension
order and its alpha and beta (as indices into the candidate sets) form the
four head labels; the features are those of the same sampled blocks.  The
network is then fitted with the library's training kernels.  Every step
runs in the CUDA library; this module only batches the calls.
"""

from __future__ import annotations

import os

import numpy as np
import torch

from . import _binding as B


def label_of(rep, alphas, betas):
    """Head labels (interpolator, order, alpha index, beta index) of a
    sampled-tuner report."""
    p = rep.params
    ia = int(np.argmin([abs(p.alpha - a) for a in alphas]))
    ib = int(np.argmin([abs(p.beta - b) for b in betas]))
    return [int(p.interp[0]), int(p.order[0]), ia, ib]


def collect(samples, opts, metric=B.METRIC_MAXERR, stream=None, cache=None):
    """samples: iterable of (field tensor, relative bound).  Returns the
    feature rows (n x 64, CUDA float32) and labels (n x 4, CUDA int32).

    cache: an .npz path.  Labels already stored there (rows in sample order)
    are reused and only the samples after them are tuned; the file is
    rewritten with all rows, so an interrupted collection resumes where it
    stopped."""
    alphas = [opts.alphas[i] for i in range(opts.n_alpha)]
    betas = [opts.betas[i] for i in range(opts.n_beta)]
    if not alphas or not betas:
        raise ValueError("labels index the candidate lists: give opts explicit alphas and betas")
    done_x, done_y = np.zeros((0, B.NFEATURES), np.float32), np.zeros((0, 4), np.int32)
    if cache is not None and os.path.exists(cache):
        d = np.load(cache)
        done_x, done_y = d["features"], d["labels"]
    feats, labels = [], []
    for i, (x, rel) in enumerate(samples):
        if i < done_x.shape[0]:
            continue
        f = torch.empty(B.NFEATURES, dtype=torch.float32, device="cuda")
        B.features(x, rel, opts, device_out=f, stream=stream)
        rep = B.tune(x, rel, metric, float("nan"), opts, stream=stream)
        feats.append(f)
        labels.append(label_of(rep, alphas, betas))
    new_x = torch.stack(feats).cpu().numpy() if feats else np.zeros((0, B.NFEATURES), np.float32)
    new_y = np.asarray(labels, dtype=np.int32).reshape(-1, 4)
    all_x, all_y = np.concatenate([done_x, new_x]), np.concatenate([done_y, new_y])
    if cache is not None and new_x.shape[0]:
        tmp = cache + ".tmp.npz"
        np.savez(tmp, features=all_x, labels=all_y)
        os.replace(tmp, cache)
    X = torch.from_numpy(all_x).cuda()
    Y = torch.from_numpy(all_y).cuda()
    return X, Y


def fit(model, X, Y, epochs=200, batch=256, lr=3e-3, seed=0):
    """Sets the model's normalisation from X, then runs Adam over shuffled
    mini-batches.  Returns the loss of each epoch's last batch."""
    Xh = X.detach().cpu().numpy().astype(np.float64)
    mean = Xh.mean(axis=0)
    sd = Xh.std(axis=0)
    sd[sd < 1e-6] = 1.0
    model.set(mean=mean.astype(np.float32), sd=sd.astype(np.float32))
    n = X.shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    for _ in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).to(X.device)
        Xs, Ys = X.index_select(0, perm).contiguous(), Y.index_select(0, perm).contiguous()
        last = None
        for b0 in range(0, n, batch):
            xb, yb = Xs[b0:b0 + batch], Ys[b0:b0 + batch]
            want = b0 + batch >= n
            last = model.train_step(xb, yb, lr, want_loss=want)
        losses.append(last)
    return losses


def accuracy(model, X, Y):
    """Fraction of rows whose argmax matches the label, per head."""
    lo = model.forward(X).cpu().numpy()
    y = Y.cpu().numpy()
    out = []
    for h, (off, n) in enumerate(B.HEADS):
        out.append(float((np.argmax(lo[:, off:off + n], axis=1) == y[:, h]).mean()))
    return out
