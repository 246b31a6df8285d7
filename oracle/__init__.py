"""CPU checker for the HMM hot path (test infrastructure only; see
``oracle/hmm_oracle.py``)."""
