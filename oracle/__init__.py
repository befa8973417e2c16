"""CPU oracle (test infrastructure only; see ``tx16_oracle``)."""
