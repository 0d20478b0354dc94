"""Learned term screening: the perceptron's weights and their training.

``load_model()`` returns the weights trained by ``train.py`` (a file in this
directory), ready for ``iqcc.iqcc_set_screening_model``.
"""
import os

import numpy as np

MODEL = os.path.join(os.path.dirname(__file__), "model_jw.npz")


def load_model(path: str = MODEL):
    d = np.load(path)
    return d["w1"], d["b1"], d["w2"], d["b2"], d["w3"], float(d["b3"])
